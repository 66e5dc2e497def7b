// lat_lform.cu -- the L = 1/H form of the scale-factor update (expansion 2).
//
// Sec. II.B notes that DEFROST evolves L = 1/H first and the scale factor from
// it, which keeps the gradient averages out of the scale-factor equation; the
// paper prints no equation for it. In program time, with h = a'/a and the
// Hubble length l = 1/h, the acceleration equation (rho + 3p = 2 sum phidot^2 -
// 2V holds no gradient term) gives
//   l' = (s + 1) + Gamma l^2,  a' = a / l,  a''/a = -s h^2 - Gamma,
//   Gamma = (8piG/(3A^2)) a^(-2r) (sum_i <(f_i' - r h f_i)^2> - <V_pr>),
// and the f coefficient of eq. scalar-evo becomes cF = r(2-r) h^2 - r Gamma.
// l lives at the momentum times, a at the field times. The kinetic average
// needs the momenta at the field time, (pi_n + pi_{n+1})/2 = u + (dt/2) cF f with
// u = pi_n + (dt/2)(cL Lap f - dV_pr/df), so the step's own cF enters it: l_{n+1}
// and cF solve the implicit midpoint equations
//   Lambda = (l_n + l_{n+1})/2, h = 1/Lambda, w = (dt/2) cF - r h,
//   Gamma = g (sum_i <(u_i + w f_i)^2> - <V_pr>),  g = (8piG/(3A^2)) a^(-2r),
//   cF = r(2-r) h^2 - r Gamma,  l_{n+1} = l_n + dt ((s + 1) + Gamma Lambda^2),
// and then a_{n+3/2} = a_{n+1/2} exp(dt / l_{n+1}) ((ln a)' = 1/l, midpoint).
//
// The sums that close these equations need the Laplacian of the fields at the
// field time, which the fused step pass (it forms the NEW fields) does not have
// at all sites, so this form costs one more read-only pass over the four state
// arrays per step (the reason the paper keeps eq. scale, whose gradient
// average comes with the Laplacian). The pass forms per site v = u + w0 f for a
// fixed guess w0 of w and reduces
//   P0 = sum_i <v_i^2>,  Q = sum_i <v_i f_i>,  F2 = sum_i <f_i^2>,  W = <V_pr>;
// for any w, sum_i <(u_i + w f_i)^2> = P0 + 2 (w - w0) Q + (w - w0)^2 F2 exactly,
// so the last block iterates the two unknowns to convergence in FP64 from
// these four numbers and writes the coefficients of the step that follows
// (read by the step kernels as they are). The guess w0 = (dt/2) cF_prev - r / l
// (the previous step's cF, the current l) keeps w - w0 small, so that no
// cancellation between the three terms costs digits.
#include <algorithm>
#include <type_traits>

#include "lat_grid.h"
#include "lat_kernels.h"
#include "lat_stencil27.cuh"

namespace lat {

namespace {

__device__ __forceinline__ size_t lidx(int n, int x, int y, int z) { return ((size_t)z * n + y) * n + x; }

template <typename T>
struct KAcc {   // compensated (Kahan) per-thread sum
    T s = T(0), c = T(0);
    __device__ __forceinline__ void add(T v)
    {
        const T y = v - c;
        const T t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// Per-step constants of the pass, from the scalars the step left: a at the new
// field time, l at the new momentum time, the previous step's cF.
struct LfConst {
    double a, ia, cL, cdom, kappa, w0;
};

__device__ inline LfConst lf_const(const Model& M, const DevScalars* sc)
{
    LfConst k;
    k.a = sc->a;
    k.ia = 1.0 / k.a;
    k.cL = apow(k.a, k.ia, -2.0 * M.s - 2.0);
    k.cdom = M.cdom0 * apow(k.a, k.ia, M.pdom);
    k.kappa = M.kappa0 * apow(k.a, k.ia, M.pint);
    k.w0 = 0.5 * M.dt * sc->cF - M.r / sc->ell;
    return k;
}

template <typename T>
struct SiteCoef {
    T kL, hdt, cdom, kap, w0;
    T bgf, bgp;   // split storage: phi = bgf + stored, its momentum = bgp + stored
    bool quartic;
};

// One site's contributions: v_i = pi_i + (dt/2)(cL Lap f_i - dV_pr/df_i) + w0 f_i,
// from the site's values as stored (Lap f_0 is that of the stored array).
template <typename T>
__device__ __forceinline__ void site_terms(const SiteCoef<T>& C, T f0, T f1, T p0, T p1, T lap0, T lap1, T& P0, T& Q,
                                           T& F2, T& W)
{
    f0 += C.bgf;   // whole phi and its momentum (unchanged when phi is stored whole)
    p0 += C.bgp;
    const T sq0 = f0 * f0, sq1 = f1 * f1;
    const T dv0 = C.cdom * (C.quartic ? sq0 * f0 : f0) + C.kap * f0 * sq1;
    const T dv1 = C.kap * sq0 * f1;
    const T v0 = (p0 + C.hdt * (C.kL * lap0 - dv0)) + C.w0 * f0;
    const T v1 = (p1 + C.hdt * (C.kL * lap1 - dv1)) + C.w0 * f1;
    P0 = v0 * v0 + v1 * v1;
    Q = v0 * f0 + v1 * f1;
    F2 = sq0 + sq1;
    W = C.cdom * (C.quartic ? T(0.25) * sq0 * sq0 : T(0.5) * sq0) + C.kap * T(0.5) * sq0 * sq1;
}

// The implicit midpoint solve of the L form from the volume averages
// S = (P0, Q, F2, W) taken with the guess w0; writes the next step's
// coefficients into the scalar block in place (every other block of the
// launch has finished reading it), or sets LAT_ENONFINITE when it does not
// converge (a recollapse through H = 0, or non-finite sums).
__device__ inline void lform_solve(const Model& M, DevScalars* sc, const double S[kSums], double w0)
{
    DevScalars& s = *sc;
    const double a = s.a, ia = 1.0 / a, dt = M.dt, r = M.r, sg = M.s, ell = s.ell;
    const double g = M.g8A2 * (1.0 / 3.0) * apow(a, ia, -2.0 * r);
    bool ok = isfinite(S[0]) && isfinite(S[1]) && isfinite(S[2]) && isfinite(S[3]) && isfinite(ell) && ell != 0.0;
    double ell_next = ell, cF = 0.0, Gam = 0.0;
    bool converged = false;
    for (int it = 0; it < 200 && ok && !converged; it++) {
        const double Lam = 0.5 * (ell + ell_next), h = 1.0 / Lam;
        const double dw = (0.5 * dt * cF - r * h) - w0;
        const double P = S[0] + 2.0 * dw * S[1] + dw * dw * S[2];
        Gam = g * (P - S[3]);
        const double cF_new = r * (2.0 - r) * h * h - r * Gam;
        const double ell_new = ell + dt * ((sg + 1.0) + Gam * Lam * Lam);
        ok = isfinite(cF_new) && isfinite(ell_new);
        // stop at 1e-13 of the size of the terms: rounding leaves a cycle of a few ulps
        converged = fabs(ell_new - ell_next) <= 1e-13 * fabs(ell_new) &&
                    fabs(cF_new - cF) <= 1e-13 * fabs(r) * (fabs(2.0 - r) * h * h + fabs(Gam));
        cF = cF_new;
        ell_next = ell_new;
    }
    if (!ok || !converged) {
        s.status = LAT_ENONFINITE;
        return;
    }
    const double h = 2.0 / (ell + ell_next);
    s.cL = apow(a, ia, -2.0 * sg - 2.0);
    s.cF = cF;
    s.cdom = M.cdom0 * apow(a, ia, M.pdom);
    s.kappa = M.kappa0 * apow(a, ia, M.pint);
    s.ad_half = a * h;
    s.add = a * (-sg * h * h - Gam);
    s.ad_next = a * expm1(dt / ell_next) / dt;   // a_{n+3/2} - a_{n+1/2} = a (exp(dt/l) - 1)
    s.ell_next = ell_next;
    step_coefficients(M, &s);
}

// Block sums into the partials; the block that finishes last folds them in a
// fixed order and runs the solve.
template <typename A>
__device__ inline void lform_finish(const Model& M, DevScalars* sc, double* partials, A v[kSums], double* red,
                                    double w0)
{
    const int nblocks = gridDim.x;
    const int tid = threadIdx.x;
    double bs[kSums];
    block_reduce(v, red, bs);
    __shared__ unsigned int is_last;
    if (tid == 0) {
        for (int k = 0; k < kSums; k++) partials[(size_t)blockIdx.x * kSums + k] = bs[k];
        __threadfence();
        is_last = atomicAdd(&sc->ticket, 1u) == (unsigned int)nblocks - 1u;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    if (tid >= 32) return;
    // lane l folds blocks l, l + 32, ... in order, the loads of four of them in
    // flight together (kSums = 4 doubles per block: two double2 loads)
    double acc[kSums] = {0.0, 0.0, 0.0, 0.0};
    const double2* p2 = reinterpret_cast<const double2*>(partials);
    int b = tid;
    for (; b + 96 < nblocks; b += 128) {
        double2 x[4][2];
#pragma unroll
        for (int j = 0; j < 4; j++) {
            x[j][0] = __ldcg(p2 + (size_t)(b + 32 * j) * 2);
            x[j][1] = __ldcg(p2 + (size_t)(b + 32 * j) * 2 + 1);
        }
#pragma unroll
        for (int j = 0; j < 4; j++) {
            acc[0] += x[j][0].x;
            acc[1] += x[j][0].y;
            acc[2] += x[j][1].x;
            acc[3] += x[j][1].y;
        }
    }
    for (; b < nblocks; b += 32) {
        const double2 x0 = __ldcg(p2 + (size_t)b * 2), x1 = __ldcg(p2 + (size_t)b * 2 + 1);
        acc[0] += x0.x;
        acc[1] += x0.y;
        acc[2] += x1.x;
        acc[3] += x1.y;
    }
#pragma unroll
    for (int k = 0; k < kSums; k++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
    if (tid == 0) {
        sc->ticket = 0u;
        double S[kSums];
        for (int k = 0; k < kSums; k++) S[k] = acc[k] * M.inv_sites;
        lform_solve(M, sc, S, w0);
        __threadfence();
    }
}

template <typename T>
__device__ inline SiteCoef<T> block_coefs(const Model& M, const DevScalars* sc, double* w0_used)
{
    __shared__ double kc[6];
    if (threadIdx.x == 0) {
        const LfConst k = lf_const(M, sc);
        kc[0] = k.cL * M.lap_scale;
        kc[1] = k.cdom;
        kc[2] = k.kappa;
        kc[3] = (double)(T)k.w0;   // the guess exactly as the sites use it
        kc[4] = sc->bgf;
        kc[5] = sc->bgp;
    }
    __syncthreads();
    SiteCoef<T> C;
    C.kL = (T)kc[0];
    C.hdt = (T)(0.5 * M.dt);
    C.cdom = (T)kc[1];
    C.kap = (T)kc[2];
    C.w0 = (T)kc[3];
    C.bgf = (T)kc[4];
    C.bgp = (T)kc[5];
    C.quartic = M.beta == 4;
    *w0_used = kc[3];
    return C;
}

// 7-point pass: one 16-byte vector (V sites along x) per thread and plane,
// marching a z run with the vectors of the planes below and above in
// registers; the y neighbours as vectors, the x neighbours beyond the vector as
// two scalars. Items: (n/V vectors x n rows) columns cut into nzc z runs.
// FP32: at most 128 registers, for 2 blocks (16 warps) per SM, each with the
// loads of two planes in flight.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1)
    lform7_kernel(Bufs<T> B, Model M, DevScalars* sc, double* partials, int nzc)
{
    constexpr int V = 16 / sizeof(T);
    using Raw = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    struct Vec {
        T v[V];
    };
    __shared__ double red[32 * kSums];
    if (sc->status != LAT_OK) return;
    double w0;
    const SiteCoef<T> C = block_coefs<T>(M, sc, &w0);
    const int n = M.n, q = n / V;
    const int par = (int)(sc->step & 1);
    const T* __restrict__ f[2] = {B.f[par][0], B.f[par][1]};
    const T* __restrict__ p[2] = {B.p[par][0], B.p[par][1]};
    KAcc<T> acc[kSums];
    auto vec = [&](const T* a, int x, int y, int z) {
        const Raw r = __ldg(reinterpret_cast<const Raw*>(a + lidx(n, x, y, z)));
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
        // what plane z needs beyond the centre vectors: the centre above (z + 1),
        // the y neighbours, the momenta and the two x neighbours past the vector
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
            o.l = __ldg(f[i] + lidx(n, xl, y, z));
            o.r = __ldg(f[i] + lidx(n, xr, y, z));
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
            // the loads of plane z + 1 go out before plane z is computed
            const Plane cu[2] = {nx[0], nx[1]};
            if (z + 1 < ze) {
#pragma unroll
                for (int i = 0; i < 2; i++) load_plane(i, z + 1, nx[i]);
            }
            Vec lap[2];
#pragma unroll
            for (int i = 0; i < 2; i++) {
#pragma unroll
                for (int j = 0; j < V; j++) {
                    const T cc = c[i].v[j];
                    const T left = j == 0 ? cu[i].l : c[i].v[j - 1], right = j == V - 1 ? cu[i].r : c[i].v[j + 1];
                    lap[i].v[j] = ((left - cc) + (right - cc)) + ((cu[i].a.v[j] - cc) + (cu[i].b.v[j] - cc)) +
                                  ((cm[i].v[j] - cc) + (cu[i].cp.v[j] - cc));
                }
            }
            T s[kSums] = {T(0), T(0), T(0), T(0)};
#pragma unroll
            for (int j = 0; j < V; j++) {
                T t[kSums];
                site_terms(C, c[0].v[j], c[1].v[j], cu[0].pv.v[j], cu[1].pv.v[j], lap[0].v[j], lap[1].v[j], t[0],
                           t[1], t[2], t[3]);
#pragma unroll
                for (int k = 0; k < kSums; k++) s[k] += t[k];
            }
#pragma unroll
            for (int k = 0; k < kSums; k++) acc[k].add(s[k]);
#pragma unroll
            for (int i = 0; i < 2; i++) {
                cm[i] = c[i];
                c[i] = cu[i].cp;
            }
        }
    }
    T v[kSums] = {acc[0].s, acc[1].s, acc[2].s, acc[3].s};
    lform_finish(M, sc, partials, v, red, w0);
}

// 27-point pass: one site per thread and plane (the weighted differences to
// all 26 neighbours in the lattice precision, exact for f = const + small).
template <typename T>
__global__ void __launch_bounds__(256) lform27_kernel(Bufs<T> B, Model M, DevScalars* sc, double* partials, int nzc)
{
    __shared__ double red[32 * kSums];
    if (sc->status != LAT_OK) return;
    double w0;
    const SiteCoef<T> C = block_coefs<T>(M, sc, &w0);
    const int n = M.n;
    const int par = (int)(sc->step & 1);
    const T* __restrict__ f0 = B.f[par][0];
    const T* __restrict__ f1 = B.f[par][1];
    const T* __restrict__ p0 = B.p[par][0];
    const T* __restrict__ p1 = B.p[par][1];
    KAcc<T> acc[kSums];
    const long long cols = (long long)n * n, items = cols * nzc;
    for (long long it = (long long)blockIdx.x * blockDim.x + threadIdx.x; it < items;
         it += (long long)gridDim.x * blockDim.x) {
        const long long col = it % cols;
        const int zc = (int)(it / cols);
        const int x = (int)(col % n), y = (int)(col / n);
        const int zb = (int)((long long)zc * n / nzc), ze = (int)((long long)(zc + 1) * n / nzc);
        for (int z = zb; z < ze; z++) {
            const size_t c = lidx(n, x, y, z);
            const T a0 = __ldg(f0 + c), a1 = __ldg(f1 + c);
            T l0 = T(0), l1 = T(0);
            for (int dz = -1; dz <= 1; dz++)
                for (int dy = -1; dy <= 1; dy++)
#pragma unroll
                    for (int dx = -1; dx <= 1; dx++) {
                        const int cls = (dx != 0) + (dy != 0) + (dz != 0);
                        if (cls == 0) continue;
                        const size_t j = lidx(n, wrap27(x + dx, n), wrap27(y + dy, n), wrap27(z + dz, n));
                        const T w = T(w27(cls));
                        l0 += w * (__ldg(f0 + j) - a0);
                        l1 += w * (__ldg(f1 + j) - a1);
                    }
            T t[kSums];
            site_terms(C, a0, a1, __ldg(p0 + c), __ldg(p1 + c), l0, l1, t[0], t[1], t[2], t[3]);
#pragma unroll
            for (int k = 0; k < kSums; k++) acc[k].add(t[k]);
        }
    }
    T v[kSums] = {acc[0].s, acc[1].s, acc[2].s, acc[3].s};
    lform_finish(M, sc, partials, v, red, w0);
}

} // namespace

template <typename T>
cudaError_t launch_lform(const Bufs<T>& b, const Model& M, DevScalars* sc, double* partials, cudaStream_t st)
{
    const int n = M.n;
    if (M.stencil == 27) {
        lform27_kernel<T><<<sums_grid_blocks(n), 256, 0, st>>>(b, M, sc, partials, sums_zruns(n));
        return cudaGetLastError();
    }
    // One resident wave of blocks (no more than the sums pass, whose partials
    // buffer this pass shares); each thread marches whole z runs, two planes
    // loaded before a run's first.
    static int occ = 0;
    const int wave = resident_wave((const void*)lform7_kernel<T>, 256, &occ);
    if (wave == 0) return cudaErrorInvalidDevice;
    constexpr int V = 16 / sizeof(T);
    const long long vcols = (long long)(n / V) * n;
    const int blocks_max = std::max(1, std::min(sums_grid_blocks(n), wave));
    const int nzc = balanced_zruns(vcols, n, (long long)blocks_max * 256, 2.0);
    const long long items = vcols * nzc;
    const int blocks = (int)std::min<long long>(blocks_max, (items + 255) / 256);
    lform7_kernel<T><<<blocks, 256, 0, st>>>(b, M, sc, partials, nzc);
    return cudaGetLastError();
}

template cudaError_t launch_lform<float>(const Bufs<float>&, const Model&, DevScalars*, double*, cudaStream_t);
template cudaError_t launch_lform<double>(const Bufs<double>&, const Model&, DevScalars*, double*, cudaStream_t);

} // namespace lat
