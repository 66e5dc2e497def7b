// lat_step_fast.cu -- the z-march step of lat_step_march.cu specialised for a
// lattice side N, a tile height TY and a prefetch depth D (planes in flight
// ahead of the one being computed) known at compile time.
//
// Same algorithm and the same results as the general kernel (Sec. II.B, eq. evo
// with eq. scalar-evo and the sums for eq. scale). With N and TY constant every
// shared-memory stride folds into an immediate offset; the ring holds RF field
// slots (D + 3 planes in use, padded so the ring period is small), RP = D + 1
// momentum slots and 2 new-field buffers, and the plane loop is unrolled by the
// period lcm(RF, RP, 2) so every slot index is a constant; and because a row of
// 16-byte vectors spans whole warps (N/4 or N/2 a multiple of 32), each warp has
// one role (halo row, owned row or look-ahead row) and its branches are uniform.
#include "lat_async.cuh"
#include "lat_kernels.h"
#include "lat_pairs.cuh"
#include "lat_site.cuh"

namespace lat {

namespace {

template <int D>
struct Ring {
    static constexpr int RF = D == 1 ? 4 : (D == 2 ? 6 : 6);   // field plane slots (>= D + 3)
    static constexpr int RP = D + 1;                           // momentum plane slots
    static constexpr int PERIOD = D == 1 ? 4 : 6;              // lcm(RF, RP, 2)
    static_assert(RF >= D + 3 && PERIOD % RF == 0 && PERIOD % RP == 0 && PERIOD % 2 == 0, "ring period");
};

template <typename T, int N, int TY, int D>
struct Fast {
    typedef typename PK<T>::P P;
    static constexpr int RF = Ring<D>::RF, RP = Ring<D>::RP, PERIOD = Ring<D>::PERIOD;
    static constexpr int NP = PK<T>::NP;
    static constexpr int VW = 2 * NP;
    static constexpr int Q = N / VW;               // vectors per row
    static constexpr int WPR = Q / 32;             // warps per row
    static constexpr int THREADS = (TY + 3) * Q;
    static constexpr uint32_t FIELDF = (TY + 3) * N, SLOTF = 2 * FIELDF;   // field slot [field][TY+3][N]
    static constexpr uint32_t FIELDP = (TY + 1) * N, SLOTP = 2 * FIELDP;   // momentum slot / new-field plane
    static constexpr uint32_t P0 = RF * SLOTF, G0 = P0 + RP * SLOTP;
    static constexpr size_t SMEM = sizeof(T) * (size_t)(G0 + 2 * SLOTP);
    static constexpr uint32_t NN = (uint32_t)N * N;
    static_assert(Q % 32 == 0, "rows must span whole warps");

    struct Ctx {
        T* S;
        uint32_t offF, offP, rowg;
        int rho, lane, z0, nz, dl, dr;
        const T *f0, *f1, *p0, *p1;
        T *of0, *of1, *op0, *op1;
        P dtcl2, dtcf2;
        SiteCoefs<T> K;
        P accg0, accg1, accvd, accvi;
    };

    static __device__ __forceinline__ void fetch_f(Ctx& C, int zrel, int slot)
    {
        const uint32_t gi = (uint32_t)wrapn(C.z0 + zrel, N) * NN + C.rowg;
        T* d = C.S + slot * SLOTF + C.offF;
        cp_async16(d, C.f0 + gi);
        cp_async16(d + FIELDF, C.f1 + gi);
    }
    static __device__ __forceinline__ void fetch_p(Ctx& C, int zrel, int slot)
    {
        const uint32_t gi = (uint32_t)wrapn(C.z0 + zrel, N) * NN + C.rowg;
        T* d = C.S + P0 + slot * SLOTP + C.offP;
        cp_async16(d, C.p0 + gi);
        cp_async16(d + FIELDP, C.p1 + gi);
    }

    // plane k = PERIOD m + J of the chunk. Field plane z0 + j lives in slot
    // (j + 1) % RF, momentum plane z0 + j in slot j % RP; plane k fetches the
    // fields of k + D + 1 and the momenta of k + D, after waiting for the group
    // committed D planes ago (fields k + 1, momenta k).
    template <int J>
    static __device__ __forceinline__ void plane(Ctx& C, int k)
    {
        const bool ahead = k == C.nz;
        const bool comp = C.rho >= 1 && C.rho <= TY + 1;   // warp-uniform
        const bool own = C.rho >= 1 && C.rho <= TY;
        cp_async_wait(D - 1);
        __syncthreads();
        if (k + D <= C.nz) {
            fetch_f(C, k + D + 1, (J + D + 2) % RF);
            if (comp) fetch_p(C, k + D, (J + D) % RP);
        }
        cp_async_commit();

        const T* Fm = C.S + (J % RF) * SLOTF;
        const T* Fc = C.S + ((J + 1) % RF) * SLOTF;
        const T* Fp = C.S + ((J + 2) % RF) * SLOTF;
        const T* Pc = C.S + P0 + (J % RP) * SLOTP;
        T* Gw = C.S + G0 + (J & 1) * SLOTP;
        const T* Gr = C.S + G0 + ((J + 1) & 1) * SLOTP;

        P cen[2][NP];
        T lefts[2], rights[2];
#pragma unroll
        for (int f = 0; f < 2; f++) {
            const T* Ff = Fc + f * FIELDF + C.offF;
            PK<T>::ld(Ff, cen[f]);
            lefts[f] = __shfl_up_sync(0xffffffffu, hi2(cen[f][NP - 1]), 1);
            rights[f] = __shfl_down_sync(0xffffffffu, lo2(cen[f][0]), 1);
            if (C.lane == 0) lefts[f] = Ff[C.dl];
            if (C.lane == 31) rights[f] = Ff[C.dr];
        }
        P g[2][NP];
        if (comp && !(ahead && C.rho == TY + 1)) {
            P pn[2][NP];
#pragma unroll
            for (int f = 0; f < 2; f++) {
                const T* Ff = Fc + f * FIELDF + C.offF;
                P up[NP], dn[NP], zm[NP], zp[NP], pv[NP], lft[NP], rgt[NP];
                PK<T>::ld(Ff - N, up);
                PK<T>::ld(Ff + N, dn);
                PK<T>::ld(Fm + f * FIELDF + C.offF, zm);
                PK<T>::ld(Fp + f * FIELDF + C.offF, zp);
                PK<T>::ld(Pc + f * FIELDP + C.offP, pv);
                if constexpr (NP == 2) {
                    T c0, c1, c2, c3;
                    un2(cen[f][0], c0, c1);
                    un2(cen[f][1], c2, c3);
                    lft[0] = mk2(lefts[f], c0);
                    lft[1] = mk2(c1, c2);
                    rgt[0] = lft[1];
                    rgt[1] = mk2(c3, rights[f]);
                } else {
                    lft[0] = mk2(lefts[f], lo2(cen[f][0]));
                    rgt[0] = mk2(hi2(cen[f][0]), rights[f]);
                }
#pragma unroll
                for (int v = 0; v < NP; v++) {
                    const P c = cen[f][v];
                    // Laplacian as a sum of neighbour differences (exact
                    // differences for f = const + small)
                    const P lapu = add2(add2(add2(sub2(lft[v], c), sub2(rgt[v], c)),
                                             add2(sub2(up[v], c), sub2(dn[v], c))),
                                        add2(sub2(zm[v], c), sub2(zp[v], c)));
                    pn[f][v] = fma2(C.dtcl2, lapu, fma2(C.dtcf2, c, pv[v]));
                }
            }
            // potential part of the kick and the drift (lat_site.cuh)
#pragma unroll
            for (int v = 0; v < NP; v++) site_kick_drift<T>(C.K, cen[0][v], cen[1][v], pn[0][v], pn[1][v], g[0][v], g[1][v]);
            if (!ahead) {
                if (own) {
                    const uint32_t gi = (uint32_t)(C.z0 + k) * NN + C.rowg;
                    PK<T>::st(C.op0 + gi, pn[0]);
                    PK<T>::st(C.op1 + gi, pn[1]);
                    PK<T>::st(C.of0 + gi, g[0]);
                    PK<T>::st(C.of1 + gi, g[1]);
                }
                PK<T>::st(Gw + C.offP, g[0]);
                PK<T>::st(Gw + FIELDP + C.offP, g[1]);
            }
        }
        // sums over the owned rows of plane k-1 (x and y pairs, potential) and
        // the z pair (k-1, k), from the new fields written one plane ago
        if (k > 0 && own) {
            P gq[2][NP];
#pragma unroll
            for (int f = 0; f < 2; f++) {
                const T* Gf = Gr + f * FIELDP + C.offP;
                P yn[NP], xn[NP];
                PK<T>::ld(Gf, gq[f]);
                PK<T>::ld(Gf + N, yn);
                T xnext = __shfl_down_sync(0xffffffffu, lo2(gq[f][0]), 1);
                if (C.lane == 31) xnext = Gf[C.dr];
                if constexpr (NP == 2) {
                    T a, b, c, d;
                    un2(gq[f][0], a, b);
                    un2(gq[f][1], c, d);
                    xn[0] = mk2(b, c);
                    xn[1] = mk2(d, xnext);
                } else {
                    xn[0] = mk2(hi2(gq[f][0]), xnext);
                }
                P acc = f == 0 ? C.accg0 : C.accg1;
#pragma unroll
                for (int v = 0; v < NP; v++) {
                    const P dxv = sub2(xn[v], gq[f][v]), dyv = sub2(yn[v], gq[f][v]), dzv = sub2(g[f][v], gq[f][v]);
                    acc = fma2(dxv, dxv, fma2(dyv, dyv, fma2(dzv, dzv, acc)));
                }
                if (f == 0) C.accg0 = acc;
                else C.accg1 = acc;
            }
#pragma unroll
            for (int v = 0; v < NP; v++) site_vsum<T>(C.K, gq[0][v], gq[1][v], C.accvd, C.accvi);
        }
    }

    // planes k + J .. k + PERIOD - 1; false once the look-ahead plane is done
    template <int J>
    static __device__ __forceinline__ bool planes(Ctx& C, int k)
    {
        plane<J>(C, k + J);
        if (k + J + 1 > C.nz) return false;
        if constexpr (J + 1 < PERIOD) return planes<J + 1>(C, k);
        else return true;
    }
};

template <typename T, int N, int TY, int D>
__global__ void __launch_bounds__(Fast<T, N, TY, D>::THREADS, (Fast<T, N, TY, D>::THREADS <= 512 ? 2 : 1))
    step_fast_kernel(Bufs<T> B, Model M, DevScalars* sc, double* partials)
{
    typedef Fast<T, N, TY, D> F;
    typedef typename F::P P;
    constexpr int VW = F::VW;
    __shared__ double red[32 * kSums];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (sc->status != LAT_OK) return;

    typename F::Ctx C;
    C.S = reinterpret_cast<T*>(smem_raw);
    const int warp = threadIdx.x >> 5;
    C.lane = threadIdx.x & 31;
    C.rho = warp / F::WPR;                                   // warp-uniform row of the tile
    const int x = ((warp - C.rho * F::WPR) * 32 + C.lane) * VW;
    C.dl = x == 0 ? N - 1 : -1;                              // left neighbour of the first site (periodic)
    C.dr = x + VW == N ? VW - N : VW;                        // right neighbour of the last site
    C.offF = (uint32_t)C.rho * N + x;
    C.offP = (uint32_t)(C.rho >= 1 && C.rho <= TY + 1 ? C.rho - 1 : 0) * N + x;
    // buffers selected with constant indices (a runtime index into the
    // parameter block would copy it to local memory)
    const bool par = (sc->step & 1) != 0;
    C.f0 = par ? B.f[1][0] : B.f[0][0];
    C.f1 = par ? B.f[1][1] : B.f[0][1];
    C.p0 = par ? B.p[1][0] : B.p[0][0];
    C.p1 = par ? B.p[1][1] : B.p[0][1];
    C.of0 = par ? B.f[0][0] : B.f[1][0];
    C.of1 = par ? B.f[0][1] : B.f[1][1];
    C.op0 = par ? B.p[0][0] : B.p[1][0];
    C.op1 = par ? B.p[0][1] : B.p[1][1];
    // f' += dt (cL Lap f + cF f - dV/df), f += dt f', with 1/dx^2 folded into dt cL
    C.K = site_coefs<T>(sc, M.beta);
    C.dtcl2 = mk2(C.K.dtcl, C.K.dtcl);
    C.dtcf2 = mk2(C.K.dtcf, C.K.dtcf);
    C.accg0 = C.accg1 = C.accvd = C.accvi = mk2(T(0), T(0));

    // Work: the (N / TY) * N (y tile, z plane) units in tile-major order; block
    // b takes units [b U / B, (b+1) U / B) and marches them as one segment per y
    // tile it touches (B = (N / TY) * c gives c balanced z chunks per tile).
    constexpr long long U = (long long)(N / TY) * N;
    long long u = (long long)blockIdx.x * U / gridDim.x;
    const long long uend = ((long long)blockIdx.x + 1) * U / gridDim.x;
    const bool comp = C.rho >= 1 && C.rho <= TY + 1;
    for (bool first = true; u < uend; first = false) {
        const int yt = (int)(u / N);
        C.z0 = (int)(u - (long long)yt * N);
        C.nz = (int)min((long long)(N - C.z0), uend - u);
        u += C.nz;
        C.rowg = (uint32_t)wrapn(yt * TY - 1 + C.rho, N) * N + x;
        // the previous segment's last plane is read by every thread before the
        // prologue refills the ring
        if (!first) __syncthreads();
        // prologue: group 0 holds field planes z0-1, z0, z0+1 and momenta z0;
        // group j (1 <= j < D) the fields of z0+1+j and the momenta of z0+j
        // (planes past the segment wrap harmlessly and go unused)
        F::fetch_f(C, -1, 0);
        F::fetch_f(C, 0, 1);
        F::fetch_f(C, 1, 2);
        if (comp) F::fetch_p(C, 0, 0);
        cp_async_commit();
#pragma unroll
        for (int j = 1; j < D; j++) {
            F::fetch_f(C, j + 1, j + 2);
            if (comp) F::fetch_p(C, j, j);
            cp_async_commit();
        }
        for (int k = 0; F::template planes<0>(C, k); k += F::PERIOD) {}
    }

    // per-thread sums in the element type (the 1/beta and 1/2 factors are
    // powers of two, exact); the block folds them as finish_block describes
    T v[kSums] = {lo2(C.accg0) + hi2(C.accg0), lo2(C.accg1) + hi2(C.accg1),
                  (lo2(C.accvd) + hi2(C.accvd)) * site_vsum_factor<T>(C.K.quartic),
                  T(0.5) * (lo2(C.accvi) + hi2(C.accvi))};
    finish_block(M, sc, partials, v, red, true);
}

// Specialised instances: (element bytes, N, TY, D).
struct FastKey {
    int esize, n, ty, depth;
};
constexpr FastKey kFast[] = {{4, 128, 4, 1}, {4, 128, 8, 1}, {4, 256, 4, 1}, {4, 256, 8, 1}, {4, 512, 2, 1},
                             {4, 512, 4, 1}, {4, 128, 8, 2}, {4, 256, 4, 2}, {4, 256, 8, 2}, {4, 512, 2, 2},
                             {8, 256, 4, 1}, {8, 512, 1, 1}};

template <typename T>
const void* fast_fn(int n, int ty, int depth, size_t* smem)
{
#define LAT_FAST_CASE(NN, TT, DD)                                  \
    if (n == NN && ty == TT && depth == DD) {                      \
        *smem = Fast<T, NN, TT, DD>::SMEM;                         \
        return (const void*)step_fast_kernel<T, NN, TT, DD>;       \
    }
    if constexpr (sizeof(T) == 4) {
        LAT_FAST_CASE(128, 4, 1) LAT_FAST_CASE(128, 8, 1) LAT_FAST_CASE(256, 4, 1) LAT_FAST_CASE(256, 8, 1)
        LAT_FAST_CASE(512, 2, 1) LAT_FAST_CASE(512, 4, 1)
        LAT_FAST_CASE(128, 8, 2) LAT_FAST_CASE(256, 4, 2) LAT_FAST_CASE(256, 8, 2) LAT_FAST_CASE(512, 2, 2)
    } else {
        LAT_FAST_CASE(256, 4, 1) LAT_FAST_CASE(512, 1, 1)
    }
#undef LAT_FAST_CASE
    return nullptr;
}

} // namespace

const void* fast_kernel(int elem_bytes, int n, int ty, int depth, size_t* smem)
{
    for (const FastKey& k : kFast)
        if (k.esize == elem_bytes && k.n == n && k.ty == ty && k.depth == depth)
            return elem_bytes == 4 ? fast_fn<float>(n, ty, depth, smem) : fast_fn<double>(n, ty, depth, smem);
    return nullptr;
}

template <typename T>
cudaError_t launch_step_fast(const Bufs<T>& b, const Model& M, DevScalars* sc, double* partials,
                             const MarchConfig& cfg, cudaStream_t st)
{
    size_t smem = 0;
    const void* fn = fast_fn<T>(M.n, cfg.ty, cfg.depth, &smem);
    if (!fn) return cudaErrorInvalidValue;
    void* args[] = {(void*)&b, (void*)&M, (void*)&sc, (void*)&partials};
    return cudaLaunchKernel(fn, dim3(cfg.blocks), dim3(cfg.threads), args, cfg.smem, st);
}

template cudaError_t launch_step_fast<float>(const Bufs<float>&, const Model&, DevScalars*, double*,
                                             const MarchConfig&, cudaStream_t);
template cudaError_t launch_step_fast<double>(const Bufs<double>&, const Model&, DevScalars*, double*,
                                              const MarchConfig&, cudaStream_t);

} // namespace lat
