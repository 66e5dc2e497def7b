// lat_step_simple.cu -- fused leapfrog step with plain (L1-cached) loads.
//
// One step of Sec. II.B, eq. evo for both fields at once, with eq. scalar-evo
// as the acceleration: 7-point Laplacian, potential derivative, kick of f',
// drift of f; then the volume sums of the NEW fields that eq. scale needs at
// the next field time: <|grad f|^2> from forward differences (equal to
// -<f Lap f> on the periodic lattice, the identity of Sec. II.B) and <V_pr>.
//
// The forward differences of the new fields need the new values one site
// beyond the tile in +x, +y and +z. The block therefore also kicks and drifts
// that one-site rim (reading only the old ping-pong buffers, which nobody
// writes during the step) without storing it. That keeps the whole step at one
// pass over memory: the sums the scale factor needs are ready when the kernel
// ends, and its last block performs the FP64 a(t) update.
//
// This kernel is the portable path (FP32 and FP64, any N % 4 == 0); the TMA
// plane-ring kernel in lat_step_tma.cu is the fast FP32/FP64 path on sm_103a.
#include <algorithm>

#include "lat_grid.h"
#include "lat_kernels.h"
#include "lat_stencil27.cuh"

namespace lat {

namespace {

template <typename T>
struct Coef {
    T cL, cF, cdom, kap, dt, idx2;
    int beta;
};

__device__ __forceinline__ size_t sidx(int n, int x, int y, int z)
{
    return ((size_t)z * n + y) * n + x;
}

// Kick and drift of both fields at one site from the old buffers:
// f'_new = f' + dt (cL Lap f + cF f - dV_pr/df), f_new = f + dt f'_new.
template <typename T>
__device__ __forceinline__ void site_update(const T* __restrict__ f0, const T* __restrict__ f1,
                                            const T* __restrict__ p0, const T* __restrict__ p1, int n, int x,
                                            int y, int z, const Coef<T>& C, T& np0, T& np1, T& g0, T& g1)
{
    const int xm = x == 0 ? n - 1 : x - 1, xp = x == n - 1 ? 0 : x + 1;
    const int ym = y == 0 ? n - 1 : y - 1, yp = y == n - 1 ? 0 : y + 1;
    const int zm = z == 0 ? n - 1 : z - 1, zp = z == n - 1 ? 0 : z + 1;
    const size_t c = sidx(n, x, y, z);
    const T a0 = __ldg(f0 + c), a1 = __ldg(f1 + c);
    // Laplacian as a sum of neighbour differences: for f = const + small each
    // difference is exact in floating point (Sterbenz), so the rounding error is
    // relative to the fluctuation, not to |f|.
    const T lap0 = (((__ldg(f0 + sidx(n, xm, y, z)) - a0) + (__ldg(f0 + sidx(n, xp, y, z)) - a0))
                  + ((__ldg(f0 + sidx(n, x, ym, z)) - a0) + (__ldg(f0 + sidx(n, x, yp, z)) - a0))
                  + ((__ldg(f0 + sidx(n, x, y, zm)) - a0) + (__ldg(f0 + sidx(n, x, y, zp)) - a0))) * C.idx2;
    const T lap1 = (((__ldg(f1 + sidx(n, xm, y, z)) - a1) + (__ldg(f1 + sidx(n, xp, y, z)) - a1))
                  + ((__ldg(f1 + sidx(n, x, ym, z)) - a1) + (__ldg(f1 + sidx(n, x, yp, z)) - a1))
                  + ((__ldg(f1 + sidx(n, x, y, zm)) - a1) + (__ldg(f1 + sidx(n, x, y, zp)) - a1))) * C.idx2;
    const T a0b = C.beta == 4 ? a0 * a0 * a0 : a0;       // f^(beta-1)
    const T dv0 = C.cdom * a0b + C.kap * a0 * a1 * a1;
    const T dv1 = C.kap * a0 * a0 * a1;
    np0 = __ldg(p0 + c) + C.dt * (C.cL * lap0 + C.cF * a0 - dv0);
    np1 = __ldg(p1 + c) + C.dt * (C.cL * lap1 + C.cF * a1 - dv1);
    g0 = a0 + C.dt * np0;
    g1 = a1 + C.dt * np1;
}

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(TX * TY) step_simple_kernel(Bufs<T> B, Model M, DevScalars* sc, double* partials,
                                                              int zr)
{
    __shared__ T g0s[TY + 1][TX + 1];
    __shared__ T g1s[TY + 1][TX + 1];
    __shared__ double red[32 * kSums];
    if (sc->status != LAT_OK) return;
    const int n = M.n;
    const int par = (int)(sc->step & 1);
    const T* __restrict__ f0 = B.f[par][0];
    const T* __restrict__ f1 = B.f[par][1];
    const T* __restrict__ p0 = B.p[par][0];
    const T* __restrict__ p1 = B.p[par][1];
    T* __restrict__ f0o = B.f[par ^ 1][0];
    T* __restrict__ f1o = B.f[par ^ 1][1];
    T* __restrict__ p0o = B.p[par ^ 1][0];
    T* __restrict__ p1o = B.p[par ^ 1][1];
    Coef<T> C;
    C.cL = (T)sc->cL; C.cF = (T)sc->cF; C.cdom = (T)sc->cdom; C.kap = (T)sc->kappa;
    C.dt = (T)M.dt; C.idx2 = (T)M.inv_dx2; C.beta = M.beta;

    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * zr;
    const int tw = min(TX, n - x0), th = min(TY, n - y0), z1 = min(z0 + zr, n);
    const int tid = threadIdx.x, lx = tid % TX, ly = tid / TX;
    const bool own = lx < tw && ly < th;
    int hx = -1, hy = -1;                 // the rim site this thread also updates
    if (tid < tw) { hx = tid; hy = th; }
    else if (tid < tw + th) { hx = tw; hy = tid - tw; }

    T acc_g0 = 0, acc_g1 = 0, acc_vd = 0, acc_vi = 0;
    T gp0 = 0, gp1 = 0;
    for (int z = z0; z <= z1; z++) {
        const int zz = z == n ? 0 : z;
        const bool ahead = z == z1;       // look-ahead plane: only the z-pairs need it
        if (own) {
            T np0, np1, g0, g1;
            site_update(f0, f1, p0, p1, n, x0 + lx, y0 + ly, zz, C, np0, np1, g0, g1);
            g0s[ly][lx] = g0; g1s[ly][lx] = g1;
            if (!ahead) {
                const size_t c = sidx(n, x0 + lx, y0 + ly, zz);
                p0o[c] = np0; p1o[c] = np1; f0o[c] = g0; f1o[c] = g1;
            }
        }
        if (!ahead && hx >= 0) {
            int x = x0 + hx, y = y0 + hy;
            if (x >= n) x -= n;
            if (y >= n) y -= n;
            T np0, np1, g0, g1;
            site_update(f0, f1, p0, p1, n, x, y, zz, C, np0, np1, g0, g1);
            g0s[hy][hx] = g0; g1s[hy][hx] = g1;
        }
        __syncthreads();
        if (own) {
            const T g0 = g0s[ly][lx], g1 = g1s[ly][lx];
            if (!ahead) {
                const T dx0 = g0s[ly][lx + 1] - g0, dy0 = g0s[ly + 1][lx] - g0;
                const T dx1 = g1s[ly][lx + 1] - g1, dy1 = g1s[ly + 1][lx] - g1;
                acc_g0 += dx0 * dx0 + dy0 * dy0;
                acc_g1 += dx1 * dx1 + dy1 * dy1;
                const T sq = g0 * g0;
                acc_vd += M.beta == 4 ? T(0.25) * sq * sq : T(0.5) * sq;
                acc_vi += T(0.5) * sq * g1 * g1;
            }
            if (z > z0) {
                const T dz0 = g0 - gp0, dz1 = g1 - gp1;
                acc_g0 += dz0 * dz0;
                acc_g1 += dz1 * dz1;
            }
            gp0 = g0; gp1 = g1;
        }
        __syncthreads();
    }
    double v[kSums] = {(double)acc_g0, (double)acc_g1, (double)acc_vd, (double)acc_vi};
    finish_block(M, sc, partials, v, red, true);
}

// Sums of the current fields (no step): the gradient averages of the configured
// stencil (forward differences for 7 points, the 13 owned weighted bonds of
// each site for 27) and the potential terms, one thread per (x, y) column
// marching z, for initialisation and after a state upload; its last block
// solves the a' update for the first step. Arithmetic in the lattice precision
// on exact neighbour differences; each thread keeps compensated (Kahan) sums,
// which the block folds in FP64 as the step kernels do.
template <typename T>
struct KSum {
    T s = T(0), c = T(0);
    __device__ __forceinline__ void add(T v)
    {
        const T y = v - c;
        const T t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

template <typename T>
__global__ void __launch_bounds__(256) sums_kernel(Bufs<T> B, Model M, DevScalars* sc, double* partials, int nzc)
{
    __shared__ double red[32 * kSums];
    const int n = M.n;
    const int par = (int)(sc->step & 1);
    const T* __restrict__ f0 = B.f[par][0];
    const T* __restrict__ f1 = B.f[par][1];
    const bool s27 = M.stencil == 27, quartic = M.beta == 4;
    KSum<T> acc[kSums];
    // work items: (x, y) columns cut into nzc z runs, so that small lattices
    // still give every SM enough threads
    const long long cols = (long long)n * n, items = cols * nzc;
    for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < items;
         it += (long long)gridDim.x * blockDim.x) {
        const long long col = it % cols;
        const int zc = (int)(it / cols);
        const int x = (int)(col % n), y = (int)(col / n);
        const int xp = x == n - 1 ? 0 : x + 1, yp = y == n - 1 ? 0 : y + 1;
        const int zb = (int)((long long)zc * n / nzc), ze = (int)((long long)(zc + 1) * n / nzc);
        T a0 = __ldg(f0 + sidx(n, x, y, zb)), a1 = __ldg(f1 + sidx(n, x, y, zb));
        for (int z = zb; z < ze; z++) {
            const int zp = z == n - 1 ? 0 : z + 1;
            const T u0 = __ldg(f0 + sidx(n, x, y, zp)), u1 = __ldg(f1 + sidx(n, x, y, zp));   // the next centre
            const T sq = a0 * a0;
            acc[2].add(quartic ? T(0.25) * sq * sq : T(0.5) * sq);
            acc[3].add(T(0.5) * sq * a1 * a1);
            if (s27) {
                acc[0].add(bonds27_sum<T>(f0, n, x, y, z));
                acc[1].add(bonds27_sum<T>(f1, n, x, y, z));
            } else {
                const T e0 = __ldg(f0 + sidx(n, xp, y, z)) - a0, e1 = __ldg(f0 + sidx(n, x, yp, z)) - a0, e2 = u0 - a0;
                const T h0 = __ldg(f1 + sidx(n, xp, y, z)) - a1, h1 = __ldg(f1 + sidx(n, x, yp, z)) - a1, h2 = u1 - a1;
                acc[0].add(e0 * e0 + e1 * e1 + e2 * e2);
                acc[1].add(h0 * h0 + h1 * h1 + h2 * h2);
            }
            a0 = u0;
            a1 = u1;
        }
    }
    T v[kSums] = {acc[0].s, acc[1].s, acc[2].s, acc[3].s};
    finish_block(M, sc, partials, v, red, false);
}

// The 7-point sums of an FP32 lattice with one 16-byte vector (four x sites)
// per thread: per plane, the vector, the one above it in y and in z, and the
// site right of its last one. Same terms and accuracy as sums_kernel; the
// vector loads keep each warp on 512 contiguous bytes of a row, and the loads of
// plane z + 1 go out before plane z is summed.
__global__ void __launch_bounds__(256) sums7_vec_kernel(Bufs<float> B, Model M, DevScalars* sc, double* partials,
                                                        int nzc)
{
    __shared__ double red[32 * kSums];
    const int n = M.n, q = n / 4;
    const int par = (int)(sc->step & 1);
    const float* __restrict__ f0 = B.f[par][0];
    const float* __restrict__ f1 = B.f[par][1];
    const bool quartic = M.beta == 4;
    KSum<float> acc[kSums];
    const long long vcols = (long long)q * n, items = vcols * nzc;
    for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < items;
         it += (long long)gridDim.x * blockDim.x) {
        const long long vc = it % vcols;
        const int zc = (int)(it / vcols);
        const int xv = (int)(vc % q), y = (int)(vc / q);
        const int x = 4 * xv, xr = x + 4 == n ? 0 : x + 4, yp = y == n - 1 ? 0 : y + 1;
        const int zb = (int)((long long)zc * n / nzc), ze = (int)((long long)(zc + 1) * n / nzc);
        auto vec = [&](const float* f, int yy, int zz) {
            return __ldg(reinterpret_cast<const float4*>(f + sidx(n, x, yy, zz)));
        };
        // per plane z: the vectors above in z and in y, the site right of the vector
        struct Plane {
            float4 u0, u1, y0, y1;
            float r0, r1;
        };
        auto load_plane = [&](int z, Plane& o) {
            const int zp = z == n - 1 ? 0 : z + 1;
            o.u0 = vec(f0, y, zp);
            o.u1 = vec(f1, y, zp);
            o.y0 = vec(f0, yp, z);
            o.y1 = vec(f1, yp, z);
            o.r0 = __ldg(f0 + sidx(n, xr, y, z));
            o.r1 = __ldg(f1 + sidx(n, xr, y, z));
        };
        float4 c0 = vec(f0, y, zb), c1 = vec(f1, y, zb);
        Plane nx;
        load_plane(zb, nx);
        for (int z = zb; z < ze; z++) {
            const Plane cu = nx;
            if (z + 1 < ze) load_plane(z + 1, nx);
            const float4 u0 = cu.u0, u1 = cu.u1, y0 = cu.y0, y1 = cu.y1;
            const float r0 = cu.r0, r1 = cu.r1;
            auto grad = [](float4 c, float4 yn, float4 zn, float r) {
                const float ex0 = c.y - c.x, ex1 = c.z - c.y, ex2 = c.w - c.z, ex3 = r - c.w;
                const float ey0 = yn.x - c.x, ey1 = yn.y - c.y, ey2 = yn.z - c.z, ey3 = yn.w - c.w;
                const float ez0 = zn.x - c.x, ez1 = zn.y - c.y, ez2 = zn.z - c.z, ez3 = zn.w - c.w;
                return ((ex0 * ex0 + ey0 * ey0 + ez0 * ez0) + (ex1 * ex1 + ey1 * ey1 + ez1 * ez1)) +
                       ((ex2 * ex2 + ey2 * ey2 + ez2 * ez2) + (ex3 * ex3 + ey3 * ey3 + ez3 * ez3));
            };
            acc[0].add(grad(c0, y0, u0, r0));
            acc[1].add(grad(c1, y1, u1, r1));
            const float s0 = c0.x * c0.x, s1 = c0.y * c0.y, s2 = c0.z * c0.z, s3 = c0.w * c0.w;
            acc[2].add(quartic ? 0.25f * ((s0 * s0 + s1 * s1) + (s2 * s2 + s3 * s3)) : 0.5f * ((s0 + s1) + (s2 + s3)));
            acc[3].add(0.5f * ((s0 * c1.x * c1.x + s1 * c1.y * c1.y) + (s2 * c1.z * c1.z + s3 * c1.w * c1.w)));
            c0 = u0;
            c1 = u1;
        }
    }
    float v[kSums] = {acc[0].s, acc[1].s, acc[2].s, acc[3].s};
    finish_block(M, sc, partials, v, red, false);
}

} // namespace

int simple_grid_blocks(int n, int zr)
{
    return ((n + kSimpleTX - 1) / kSimpleTX) * ((n + kSimpleTY - 1) / kSimpleTY) * ((n + zr - 1) / zr);
}

template <typename T>
cudaError_t launch_step_simple(const Bufs<T>& b, const Model& M, DevScalars* sc, double* partials, int zr,
                               cudaStream_t st)
{
    const int n = M.n;
    dim3 grid((n + kSimpleTX - 1) / kSimpleTX, (n + kSimpleTY - 1) / kSimpleTY, (n + zr - 1) / zr);
    step_simple_kernel<T, kSimpleTX, kSimpleTY><<<grid, kSimpleTX * kSimpleTY, 0, st>>>(b, M, sc, partials, zr);
    return cudaGetLastError();
}

// z runs per (x, y) column of the sums pass: about 4 x 152 x 256 threads'
// worth of (column, run) items, runs of at least 4 planes
int sums_zruns(int n)
{
    const long long cols = (long long)n * n;
    return (int)std::max<long long>(1, std::min<long long>(n / 4, (155648 + cols - 1) / cols));
}

int sums_grid_blocks(int n)
{
    const long long items = (long long)n * n * sums_zruns(n);
    long long blocks = (items + 255) / 256;
    return (int)(blocks < 1024 ? blocks : 1024);
}

template <typename T>
cudaError_t launch_sums(const Bufs<T>& b, const Model& M, DevScalars* sc, double* partials, cudaStream_t st)
{
    if constexpr (sizeof(T) == 4) {
        if (M.stencil != 27) {
            // vector items: (n/4 vectors x n rows) columns cut into z runs. One
            // resident wave of blocks (no more than sums_grid_blocks, which sizes the
            // partials buffer); each thread marches whole runs, one plane loaded
            // before a run's first.
            static int occ = 0;
            const int wave = resident_wave((const void*)sums7_vec_kernel, 256, &occ);
            if (wave == 0) return cudaErrorInvalidDevice;
            const int n = M.n;
            const long long vcols = (long long)(n / 4) * n;
            const int blocks_max = std::max(1, std::min(sums_grid_blocks(n), wave));
            const int nzc = balanced_zruns(vcols, n, (long long)blocks_max * 256, 1.0);
            const long long items = vcols * nzc;
            const int blocks = (int)std::min<long long>(blocks_max, (items + 255) / 256);
            sums7_vec_kernel<<<blocks, 256, 0, st>>>(b, M, sc, partials, nzc);
            return cudaGetLastError();
        }
    }
    sums_kernel<T><<<sums_grid_blocks(M.n), 256, 0, st>>>(b, M, sc, partials, sums_zruns(M.n));
    return cudaGetLastError();
}

template cudaError_t launch_step_simple<float>(const Bufs<float>&, const Model&, DevScalars*, double*, int,
                                               cudaStream_t);
template cudaError_t launch_step_simple<double>(const Bufs<double>&, const Model&, DevScalars*, double*, int,
                                                cudaStream_t);
template cudaError_t launch_sums<float>(const Bufs<float>&, const Model&, DevScalars*, double*, cudaStream_t);
template cudaError_t launch_sums<double>(const Bufs<double>&, const Model&, DevScalars*, double*, cudaStream_t);

} // namespace lat
