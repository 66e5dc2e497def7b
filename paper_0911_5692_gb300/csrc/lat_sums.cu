// lat_sums.cu -- the volume averages of the current fields without a step
// (after initialisation, a state upload or a change of coupling): the gradient
// averages <|grad f|^2> = -<f L f> of the configured stencil (Sec. II.B, the
// divergence-theorem identity) and the potential terms, whose last block then
// solves the a' update of the first step (eq. scale).
#include <algorithm>

#include "lat_grid.h"
#include "lat_kernels.h"
#include "lat_site.cuh"
#include "lat_stencil27.cuh"

namespace lat {

namespace {

__device__ __forceinline__ size_t sidx(int n, int x, int y, int z)
{
    return ((size_t)z * n + y) * n + x;
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
    const T P = (T)sc->bgf, P2 = (T)(sc->bgf * sc->bgf), vfac = site_vsum_factor<T>(quartic);
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
            // potential terms about the homogeneous mode (lat_site.cuh)
            acc[2].add(vfac * vdiff_dom(a0, P, P2, quartic));
            acc[3].add(T(0.5) * vint(a0, a1, P));
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
    const float P = (float)sc->bgf, P2 = (float)(sc->bgf * sc->bgf), vfac = site_vsum_factor<float>(quartic);
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
            // potential terms about the homogeneous mode (lat_site.cuh)
            acc[2].add(vfac * ((vdiff_dom(c0.x, P, P2, quartic) + vdiff_dom(c0.y, P, P2, quartic)) +
                               (vdiff_dom(c0.z, P, P2, quartic) + vdiff_dom(c0.w, P, P2, quartic))));
            acc[3].add(0.5f * ((vint(c0.x, c1.x, P) + vint(c0.y, c1.y, P)) + (vint(c0.z, c1.z, P) + vint(c0.w, c1.w, P))));
            c0 = u0;
            c1 = u1;
        }
    }
    float v[kSums] = {acc[0].s, acc[1].s, acc[2].s, acc[3].s};
    finish_block(M, sc, partials, v, red, false);
}

} // namespace

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

template cudaError_t launch_sums<float>(const Bufs<float>&, const Model&, DevScalars*, double*, cudaStream_t);
template cudaError_t launch_sums<double>(const Bufs<double>&, const Model&, DevScalars*, double*, cudaStream_t);

} // namespace lat
