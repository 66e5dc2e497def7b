// lat_diag.cu -- diagnostics off the timed path: energy density and pressure
// parts (Sec. II.B, eq. rho-pres) and the shell-binned power spectrum that
// Sec. IV names as future work.
#include <cufft.h>

#include <algorithm>
#include <type_traits>

#include "lat_grid.h"
#include "lat_kernels.h"
#include "lat_stencil27.cuh"

namespace lat {

namespace {

__device__ __forceinline__ size_t sidx(int n, int x, int y, int z) { return ((size_t)z * n + y) * n + x; }

// Per-block FP64 partials (one thread per (x, y) column, z marched in order):
// pass 0: [kin0, kin1, grad0, grad1, pot, sum f0, sum f1], where the momenta at
// the field time are f' + (dt/2) F(f) (the average of the stored f' and the
// next kick's), kin_i = (f'_i - r h f_i)^2 / 2 with h = a'/a at the field time,
// grad_i = the stencil's gradient sum before its factor M.lap_scale (7 points:
// sum_d (forward difference)^2; 27 points: the 13 owned weighted bonds),
// pot = V_pr;
// pass 1: [0, 0, 0, 0, 0, sum (f0 - mean0)^2, sum (f1 - mean1)^2].
template <typename T>
__global__ void __launch_bounds__(256) energies_kernel(Bufs<T> B, Model M, const DevScalars* sc, double* partials,
                                                       const double* means, int pass)
{
    __shared__ double red[32][kEnergySums];
    const int n = M.n;
    const int par = (int)(sc->step & 1);
    const T* f0 = B.f[par][0];
    const T* f1 = B.f[par][1];
    const T* p0 = B.p[par][0];
    const T* p1 = B.p[par][1];
    const double cL = sc->cL, cF = sc->cF, cdom = sc->cdom, kap = sc->kappa, dt = M.dt;
    const double h = M.expansion ? sc->ad_half / sc->a : 0.0;
    // split storage: phi = P + stored, its momentum = Pi + stored (P = Pi = 0 otherwise)
    const double bgf = sc->bgf, bgp = sc->bgp;
    double acc[kEnergySums] = {0, 0, 0, 0, 0, 0, 0};
    const long long cols = (long long)n * n;
    for (long long col = (long long)blockIdx.x * blockDim.x + threadIdx.x; col < cols;
         col += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(col % n), y = (int)(col / n);
        const int xm = x == 0 ? n - 1 : x - 1, xp = x == n - 1 ? 0 : x + 1;
        const int ym = y == 0 ? n - 1 : y - 1, yp = y == n - 1 ? 0 : y + 1;
        for (int z = 0; z < n; z++) {
            const size_t c = sidx(n, x, y, z);
            const double s0 = (double)f0[c], a1 = (double)f1[c];
            const double a0 = s0 + bgf;
            if (pass == 1) {
                const double d0 = a0 - means[0], d1 = a1 - means[1];
                acc[5] += d0 * d0;
                acc[6] += d1 * d1;
                continue;
            }
            const int zm = z == 0 ? n - 1 : z - 1, zp = z == n - 1 ? 0 : z + 1;
            double lap0, lap1, gs0, gs1;
            if (M.stencil == 27) {
                lap0 = lap27_sum(f0, n, x, y, z) * M.lap_scale;
                lap1 = lap27_sum(f1, n, x, y, z) * M.lap_scale;
                gs0 = bonds27_sum(f0, n, x, y, z);
                gs1 = bonds27_sum(f1, n, x, y, z);
            } else {
                const double fx0 = (double)f0[sidx(n, xp, y, z)], fy0 = (double)f0[sidx(n, x, yp, z)],
                             fz0 = (double)f0[sidx(n, x, y, zp)];
                const double fx1 = (double)f1[sidx(n, xp, y, z)], fy1 = (double)f1[sidx(n, x, yp, z)],
                             fz1 = (double)f1[sidx(n, x, y, zp)];
                lap0 = (((fx0 - s0) + ((double)f0[sidx(n, xm, y, z)] - s0)) + ((fy0 - s0) + ((double)f0[sidx(n, x, ym, z)] - s0))
                                     + ((fz0 - s0) + ((double)f0[sidx(n, x, y, zm)] - s0))) * M.inv_dx2;
                lap1 = (((fx1 - a1) + ((double)f1[sidx(n, xm, y, z)] - a1)) + ((fy1 - a1) + ((double)f1[sidx(n, x, ym, z)] - a1))
                                     + ((fz1 - a1) + ((double)f1[sidx(n, x, y, zm)] - a1))) * M.inv_dx2;
                gs0 = (fx0 - s0) * (fx0 - s0) + (fy0 - s0) * (fy0 - s0) + (fz0 - s0) * (fz0 - s0);
                gs1 = (fx1 - a1) * (fx1 - a1) + (fy1 - a1) * (fy1 - a1) + (fz1 - a1) * (fz1 - a1);
            }
            const double a0b = M.beta == 4 ? a0 * a0 * a0 : a0;
            const double F0 = cL * lap0 + cF * a0 - (cdom * a0b + kap * a0 * a1 * a1);
            const double F1 = cL * lap1 + cF * a1 - kap * a0 * a0 * a1;
            const double q0 = ((double)p0[c] + bgp) + 0.5 * dt * F0 - M.r * h * a0;
            const double q1 = (double)p1[c] + 0.5 * dt * F1 - M.r * h * a1;
            acc[0] += 0.5 * q0 * q0;
            acc[1] += 0.5 * q1 * q1;
            acc[2] += gs0;
            acc[3] += gs1;
            const double sq = a0 * a0;
            acc[4] += cdom * (M.beta == 4 ? 0.25 * sq * sq : 0.5 * sq) + 0.5 * kap * sq * a1 * a1;
            acc[5] += a0;
            acc[6] += a1;
        }
    }
    // deterministic block reduction: shuffle tree, then warp totals in order
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int k = 0; k < kEnergySums; k++) {
        for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
        if (lane == 0) red[warp][k] = acc[k];
    }
    __syncthreads();
    if (threadIdx.x < kEnergySums) {
        double s = 0.0;
        for (int w = 0; w < nwarps; w++) s += red[w][threadIdx.x];
        partials[(size_t)blockIdx.x * kEnergySums + threadIdx.x] = s;
    }
}

template <typename T>
__global__ void to_double_kernel(const T* src, double* dst, size_t count)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        dst[i] = (double)src[i];
}

// Shell binning of the R2C half spectrum ([kz][ky][kx], kx in [0, N/2]). Modes
// with 0 < kx < N/2 stand for themselves and their conjugate partner (weight 2).
// Each block accumulates into shared-memory bins and writes its own row of
// partials [p(nbins), k(nbins), count(nbins)]; the host folds the rows in block
// order.
__global__ void spectrum_bins_kernel(const cufftDoubleComplex* spec, int n, double L, int nbins, double* partials)
{
    extern __shared__ double sb[];
    for (int i = threadIdx.x; i < 3 * nbins; i += blockDim.x) sb[i] = 0.0;
    __syncthreads();
    const int nh = n / 2 + 1;
    const size_t count = (size_t)n * n * nh;
    const double inv_n3 = 1.0 / ((double)n * n * n);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const int kx = (int)(i % nh);
        const int ky = (int)((i / nh) % n);
        const int kz = (int)(i / ((size_t)nh * n));
        const int nx = kx < n / 2 ? kx : kx - n;
        const int ny = ky < n / 2 ? ky : ky - n;
        const int nz = kz < n / 2 ? kz : kz - n;
        const double nmag = sqrt((double)nx * nx + (double)ny * ny + (double)nz * nz);
        const int b = (int)floor(nmag + 0.5);
        if (b >= nbins) continue;
        const double w = (kx == 0 || 2 * kx == n) ? 1.0 : 2.0;
        const double pw = (spec[i].x * spec[i].x + spec[i].y * spec[i].y) * inv_n3;
        atomicAdd(&sb[b], w * pw);
        atomicAdd(&sb[nbins + b], w * 2.0 * 3.14159265358979323846 * nmag / L);
        atomicAdd(&sb[2 * nbins + b], w);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * nbins; i += blockDim.x) partials[(size_t)blockIdx.x * 3 * nbins + i] = sb[i];
}

// Integer-weight sums over the site's stencil neighbours of the differences
// (30 dx^2 L f for 27 points, dx^2 L f for 7) and of their squares.
template <typename T>
__device__ __forceinline__ void neighbour_sums(const T* __restrict__ f, int n, int x, int y, int z, bool s27, T& lap,
                                               T& sq)
{
    const T c = __ldg(f + sidx(n, x, y, z));
    T l = T(0), g = T(0);
    if (s27) {
#pragma unroll
        for (int dz = -1; dz <= 1; dz++) {
            const int zz = wrap27(z + dz, n);
#pragma unroll
            for (int dy = -1; dy <= 1; dy++) {
                const int yy = wrap27(y + dy, n);
#pragma unroll
                for (int dx = -1; dx <= 1; dx++) {
                    const int cls = (dx != 0) + (dy != 0) + (dz != 0);
                    if (cls == 0) continue;
                    const T d = __ldg(f + sidx(n, wrap27(x + dx, n), yy, zz)) - c;
                    const T w = T(w27(cls));
                    l += w * d;
                    g += w * d * d;
                }
            }
        }
    } else {
        const int xm = x == 0 ? n - 1 : x - 1, xp = x == n - 1 ? 0 : x + 1;
        const int ym = y == 0 ? n - 1 : y - 1, yp = y == n - 1 ? 0 : y + 1;
        const int zm = z == 0 ? n - 1 : z - 1, zp = z == n - 1 ? 0 : z + 1;
        const T d[6] = {__ldg(f + sidx(n, xm, y, z)) - c, __ldg(f + sidx(n, xp, y, z)) - c,
                        __ldg(f + sidx(n, x, ym, z)) - c, __ldg(f + sidx(n, x, yp, z)) - c,
                        __ldg(f + sidx(n, x, y, zm)) - c, __ldg(f + sidx(n, x, y, zp)) - c};
#pragma unroll
        for (int k = 0; k < 6; k++) {
            l += d[k];
            g += d[k] * d[k];
        }
    }
    lap = l;
    sq = g;
}

// Energy density and pressure at every site (eq. rho-pres per site), in the
// units of lat_energies: rho = conv (sum_i [kin_i + grad_i] + V_pr),
// p = conv (sum_i [kin_i - grad_i / 3] - V_pr), kin_i = (f'_i + (dt/2) F_i - r h f_i)^2 / 2
// (the momentum at the field time), grad_i = a^(-2s-2) / 2 times half the
// weighted squared differences to all the site's stencil neighbours (each
// neighbour pair shared evenly by its two sites). One thread per (x, y) column;
// arithmetic in the lattice precision on exact neighbour differences, the
// coefficients in FP64 rounded once.
template <typename T>
struct FieldCoef {
    T cL, cF, cdom, kap, hdt, rh, gq, cv;
    T bgf, bgp;   // split storage: phi = bgf + stored, its momentum = bgp + stored
    bool quartic;
};

template <typename T>
__device__ inline FieldCoef<T> field_coefs(const Model& M, const DevScalars* sc)
{
    const double a = sc->a;
    const double h = M.expansion ? sc->ad_half / a : 0.0;
    FieldCoef<T> k;
    k.cL = (T)(sc->cL * M.lap_scale);
    k.cF = (T)sc->cF;
    k.cdom = (T)sc->cdom;
    k.kap = (T)sc->kappa;
    k.hdt = (T)(0.5 * M.dt);
    k.rh = (T)(M.r * h);
    k.gq = (T)(0.25 * pow(a, -2.0 * M.s - 2.0) * M.lap_scale);   // grad_i = gq * sum w d^2
    k.cv = (T)(M.B * M.B / (M.A * M.A) * pow(a, 2.0 * M.s - 2.0 * M.r));
    k.bgf = (T)sc->bgf;
    k.bgp = (T)sc->bgp;
    k.quartic = M.beta == 4;
    return k;
}

// rho and p at one site from its fields a0, a1, momenta m0, m1 as stored and
// the neighbour sums (l: of the differences, g: of their squares) of each field.
template <typename T>
__device__ __forceinline__ void site_energy(const FieldCoef<T>& K, T a0, T a1, T m0, T m1, T l0, T g0, T l1, T g1,
                                            T& rho, T& pres)
{
    a0 += K.bgf;   // whole phi and its momentum (unchanged when phi is stored whole)
    m0 += K.bgp;
    const T a0b = K.quartic ? a0 * a0 * a0 : a0;
    const T F0 = K.cL * l0 + K.cF * a0 - (K.cdom * a0b + K.kap * a0 * a1 * a1);
    const T F1 = K.cL * l1 + K.cF * a1 - K.kap * a0 * a0 * a1;
    const T q0 = m0 + K.hdt * F0 - K.rh * a0;
    const T q1 = m1 + K.hdt * F1 - K.rh * a1;
    const T kin = T(0.5) * (q0 * q0 + q1 * q1);
    const T grad = K.gq * (g0 + g1);
    const T sq = a0 * a0;
    const T V = K.cdom * (K.quartic ? T(0.25) * sq * sq : T(0.5) * sq) + T(0.5) * K.kap * sq * a1 * a1;
    rho = K.cv * (kin + grad + V);
    pres = K.cv * (kin - grad / T(3) - V);
}

template <typename T>
__global__ void __launch_bounds__(256) energy_field_kernel(Bufs<T> B, Model M, const DevScalars* sc, T* rho, T* pres)
{
    const int n = M.n;
    const int par = (int)(sc->step & 1);
    const T* f0 = B.f[par][0];
    const T* f1 = B.f[par][1];
    const T* p0 = B.p[par][0];
    const T* p1 = B.p[par][1];
    const FieldCoef<T> K = field_coefs<T>(M, sc);
    const bool s27 = M.stencil == 27;
    const long long cols = (long long)n * n;
    for (long long col = (long long)blockIdx.x * blockDim.x + threadIdx.x; col < cols;
         col += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(col % n), y = (int)(col / n);
        for (int z = 0; z < n; z++) {
            const size_t c = sidx(n, x, y, z);
            const T a0 = __ldg(f0 + c), a1 = __ldg(f1 + c);
            T l0, g0, l1, g1;
            neighbour_sums(f0, n, x, y, z, s27, l0, g0);
            neighbour_sums(f1, n, x, y, z, s27, l1, g1);
            site_energy(K, a0, a1, __ldg(p0 + c), __ldg(p1 + c), l0, g0, l1, g1, rho[c], pres[c]);
        }
    }
}

// The 7-point energy field with one 16-byte vector of x sites per thread,
// marching whole z runs, the loads of plane z + 1 issued before plane z is
// computed; the same per-site terms as energy_field_kernel, the six neighbour
// differences taken in the same order (-x, +x, -y, +y, -z, +z).
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1)
    energy_field7_kernel(Bufs<T> B, Model M, const DevScalars* sc, T* rho, T* pres, int nzc)
{
    constexpr int V = 16 / sizeof(T);
    using Raw = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    struct Vec {
        T v[V];
    };
    const int n = M.n, q = n / V;
    const int par = (int)(sc->step & 1);
    const T* __restrict__ f[2] = {B.f[par][0], B.f[par][1]};
    const T* __restrict__ p[2] = {B.p[par][0], B.p[par][1]};
    const FieldCoef<T> K = field_coefs<T>(M, sc);
    auto vec = [&](const T* a, int x, int y, int z) {
        const Raw r = __ldg(reinterpret_cast<const Raw*>(a + sidx(n, x, y, z)));
        Vec o;
        *reinterpret_cast<Raw*>(o.v) = r;
        return o;
    };
    const long long vcols = (long long)q * n, items = vcols * nzc;
    for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < items;
         it += (long long)gridDim.x * blockDim.x) {
        const long long vc = it % vcols;
        const int zc = (int)(it / vcols);
        const int x = V * (int)(vc % q), y = (int)(vc / q);
        const int xl = x == 0 ? n - 1 : x - 1, xr = x + V == n ? 0 : x + V;
        const int ym = y == 0 ? n - 1 : y - 1, yp = y == n - 1 ? 0 : y + 1;
        const int zb = (int)((long long)zc * n / nzc), ze = (int)((long long)(zc + 1) * n / nzc);
        struct Plane {
            Vec cp, a, b, pv;
            T l, r;
        };
        auto load_plane = [&](int i, int z, Plane& o) {
            const int zp = z == n - 1 ? 0 : z + 1;
            o.cp = vec(f[i], x, y, zp);
            o.a = vec(f[i], x, ym, z);
            o.b = vec(f[i], x, yp, z);
            o.pv = vec(p[i], x, y, z);
            o.l = __ldg(f[i] + sidx(n, xl, y, z));
            o.r = __ldg(f[i] + sidx(n, xr, y, z));
        };
        Vec cm[2], c[2];
        Plane nx[2];
#pragma unroll
        for (int i = 0; i < 2; i++) {
            cm[i] = vec(f[i], x, y, zb == 0 ? n - 1 : zb - 1);
            c[i] = vec(f[i], x, y, zb);
            load_plane(i, zb, nx[i]);
        }
        for (int z = zb; z < ze; z++) {
            const Plane cu[2] = {nx[0], nx[1]};
            if (z + 1 < ze) {
#pragma unroll
                for (int i = 0; i < 2; i++) load_plane(i, z + 1, nx[i]);
            }
            Vec lsum[2], gsum[2];
#pragma unroll
            for (int i = 0; i < 2; i++) {
#pragma unroll
                for (int j = 0; j < V; j++) {
                    const T cc = c[i].v[j];
                    const T left = j == 0 ? cu[i].l : c[i].v[j - 1], right = j == V - 1 ? cu[i].r : c[i].v[j + 1];
                    const T d[6] = {left - cc, right - cc, cu[i].a.v[j] - cc, cu[i].b.v[j] - cc, cm[i].v[j] - cc,
                                    cu[i].cp.v[j] - cc};
                    T l = T(0), g = T(0);
#pragma unroll
                    for (int k = 0; k < 6; k++) {
                        l += d[k];
                        g += d[k] * d[k];
                    }
                    lsum[i].v[j] = l;
                    gsum[i].v[j] = g;
                }
            }
            Vec ro, pr;
#pragma unroll
            for (int j = 0; j < V; j++)
                site_energy(K, c[0].v[j], c[1].v[j], cu[0].pv.v[j], cu[1].pv.v[j], lsum[0].v[j], gsum[0].v[j],
                            lsum[1].v[j], gsum[1].v[j], ro.v[j], pr.v[j]);
            const size_t o = sidx(n, x, y, z);
            *reinterpret_cast<Raw*>(rho + o) = *reinterpret_cast<const Raw*>(ro.v);
            *reinterpret_cast<Raw*>(pres + o) = *reinterpret_cast<const Raw*>(pr.v);
#pragma unroll
            for (int i = 0; i < 2; i++) {
                cm[i] = c[i];
                c[i] = cu[i].cp;
            }
        }
    }
}

} // namespace

template <typename T>
cudaError_t launch_energy_field(const Bufs<T>& b, const Model& M, const DevScalars* sc, T* rho, T* pres,
                                cudaStream_t st)
{
    const int n = M.n;
    constexpr int V = 16 / sizeof(T);
    if (M.stencil != 27 && ((uintptr_t)rho % 16) == 0 && ((uintptr_t)pres % 16) == 0) {
        // one resident wave; runs of whole planes per thread, two planes loaded
        // before a run's first
        static int occ = 0;
        const int wave = resident_wave((const void*)energy_field7_kernel<T>, 256, &occ);
        if (wave == 0) return cudaErrorInvalidDevice;
        const long long vcols = (long long)(n / V) * n;
        const int nzc = balanced_zruns(vcols, n, (long long)wave * 256, 2.0);
        const int blocks = (int)std::min<long long>(wave, (vcols * nzc + 255) / 256);
        energy_field7_kernel<T><<<blocks, 256, 0, st>>>(b, M, sc, rho, pres, nzc);
        return cudaGetLastError();
    }
    energy_field_kernel<T><<<energies_grid_blocks(n), 256, 0, st>>>(b, M, sc, rho, pres);
    return cudaGetLastError();
}
template cudaError_t launch_energy_field<float>(const Bufs<float>&, const Model&, const DevScalars*, float*, float*,
                                                cudaStream_t);
template cudaError_t launch_energy_field<double>(const Bufs<double>&, const Model&, const DevScalars*, double*,
                                                 double*, cudaStream_t);

int energies_grid_blocks(int n)
{
    const long long cols = (long long)n * n;
    long long blocks = (cols + 255) / 256;
    return (int)(blocks < 1024 ? blocks : 1024);
}

template <typename T>
cudaError_t launch_energies(const Bufs<T>& b, const Model& M, const DevScalars* sc, double* partials,
                            const double* means, int pass, cudaStream_t st)
{
    energies_kernel<T><<<energies_grid_blocks(M.n), 256, 0, st>>>(b, M, sc, partials, means, pass);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_to_double(const T* src, double* dst, size_t count, cudaStream_t st)
{
    size_t blocks = (count + 255) / 256;
    to_double_kernel<T><<<(int)(blocks < 4096 ? blocks : 4096), 256, 0, st>>>(src, dst, count);
    return cudaGetLastError();
}

int spectrum_grid_blocks(int n)
{
    const size_t count = (size_t)n * n * (n / 2 + 1);
    size_t blocks = (count + 255) / 256;
    return (int)(blocks < 256 ? blocks : 256);
}

cudaError_t launch_spectrum_bins(const void* spec, int n, double L, int nbins, double* partials, cudaStream_t st)
{
    const size_t smem = (size_t)3 * nbins * sizeof(double);
    if (smem > 48 * 1024) {
        cudaError_t e = allow_dynamic_smem((const void*)spectrum_bins_kernel, smem);
        if (e != cudaSuccess) return e;
    }
    spectrum_bins_kernel<<<spectrum_grid_blocks(n), 256, smem, st>>>((const cufftDoubleComplex*)spec, n, L, nbins,
                                                                     partials);
    return cudaGetLastError();
}

template cudaError_t launch_energies<float>(const Bufs<float>&, const Model&, const DevScalars*, double*,
                                            const double*, int, cudaStream_t);
template cudaError_t launch_energies<double>(const Bufs<double>&, const Model&, const DevScalars*, double*,
                                             const double*, int, cudaStream_t);
template cudaError_t launch_to_double<float>(const float*, double*, size_t, cudaStream_t);
template cudaError_t launch_to_double<double>(const double*, double*, size_t, cudaStream_t);

} // namespace lat
