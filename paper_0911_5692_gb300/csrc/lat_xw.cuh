// lat_xw.cuh -- the fused 7-point step over x tiles one warp wide
// (variant 5), with the lattice side N, the tile height TY and the prefetch
// depth D known at compile time.
//
// The same step as the other plane-ring kernels (Sec. II.B, eq. evo with eq.
// scalar-evo; the sums of the new fields for eq. scale from the +y row and +z
// plane look-ahead; the FP64 a(t) update in the last block). A tile is W = 32
// 16-byte vectors wide (128 FP32 or 64 FP64 columns) and TY rows tall, so every
// staged row of the tile is exactly one warp: warp r stages and computes row r
// (0: the halo row below, 1..TY: the owned rows, TY + 1: the look-ahead row,
// TY + 2: the halo row above), and every branch on a row's role is uniform
// across the warp. The tile's two columns of x neighbours are not staged as
// vectors; one more warp (the edge warp) stages, per row and plane, the scalars
// the tile needs from its x neighbours: f at x0 - 1 (left Laplacian neighbour
// of lane 0), x0 + W (right neighbour of lane 31) and x0 + W + 1, and the
// momenta at x0 + W. From them it kicks and drifts the boundary column x0 + W
// of the owned rows, rounded exactly as the neighbouring tile's own kernel
// rounds the same sites, for the x differences of the sums. With N, TY and D
// constant every shared-memory stride is an immediate and the plane loop is
// unrolled by the ring period, so the slot indices are constants.
//
// The NXT = N / W x tiles of a y tile are taken by NXT consecutive blocks that
// march the same (y tile, z plane) units at the same time, so the scalars one
// tile reads from its neighbours' columns lie in memory lines the neighbouring
// blocks are reading too (L2 hits); and neighbouring y tiles are marched at the
// same planes at the same time (lat_layout.cuh), so that a tile's halo rows,
// its neighbours' owned rows, are L2 hits too. The new state is written with
// streaming stores: only the next step reads it.
//
// SLAB instances step z ranges of the owned planes of one or several z-slabs
// (stored planes with their halos, no wrap in z; each slab with its own
// arrays), laid end to end in z for the block layout, and write the ranges'
// summed shares of the volume averages instead of advancing the scalars
// (lat_slab.cu).
#pragma once

#include <algorithm>

#include "lat_async.cuh"
#include "lat_layout.cuh"
#include "lat_kernels.h"
#include "lat_pairs.cuh"
#include "lat_site.cuh"

namespace lat {

namespace xw {

enum { kOwn, kAhead, kStage, kEdge };   // warp roles

template <int D>
struct RingXW {
    static constexpr int RF = D == 1 ? 4 : 6;          // field plane slots (>= D + 3)
    static constexpr int RP = D + 1;                   // momentum plane slots
    static constexpr int PERIOD = D == 1 ? 4 : 6;      // lcm(RF, RP, 2)
    static_assert(RF >= D + 3 && PERIOD % RF == 0 && PERIOD % RP == 0 && PERIOD % 2 == 0, "ring period");
};

template <typename T, int N, int TY, int D, bool SLAB>
struct XW {
    typedef typename PK<T>::P P;
    static constexpr int RF = RingXW<D>::RF, RP = RingXW<D>::RP, PERIOD = RingXW<D>::PERIOD;
    static constexpr int NP = PK<T>::NP;
    static constexpr int VW = 2 * NP;                  // elements per 16-byte vector
    static constexpr int W = 32 * VW;                  // tile width: one warp of vectors
    static constexpr int NXT = N / W;                  // x tiles per row
    static constexpr int ROWS = TY + 3;                // staged rows (one warp each)
    static constexpr int THREADS = (ROWS + 1) * 32;    // and the edge warp
    static_assert(N % W == 0 && N % TY == 0 && ROWS <= 32, "tile geometry");
    // shared memory, in elements: the field ring [slot][field][ROWS][W], the
    // momentum ring [slot][field][TY + 1][W], two new-field planes
    // [buf][field][TY + 1][W]; then the edge scalars: fields [slot][field][ROWS][4]
    // (x0 - 1, x0 + W, x0 + W + 1, unused), momenta [slot][field][TY] at x0 + W,
    // new fields [buf][field][TY] at x0 + W
    static constexpr uint32_t FIELDF = ROWS * W, SLOTF = 2 * FIELDF;
    static constexpr uint32_t FIELDP = (TY + 1) * W, SLOTP = 2 * FIELDP;
    static constexpr uint32_t P0 = RF * SLOTF, G0 = P0 + RP * SLOTP;
    static constexpr uint32_t EF = ROWS * 4, ESF = 2 * EF;
    static constexpr uint32_t EPF = TY, ESP = 2 * EPF;
    static constexpr uint32_t EF0 = G0 + 2 * SLOTP, EP0 = EF0 + RF * ESF, EG0 = EP0 + RP * ESP;
    static constexpr uint32_t END = EG0 + 2 * 2 * TY;
    static constexpr size_t SMEM = (sizeof(T) * (size_t)END + 15) / 16 * 16;
    static constexpr uint32_t NN = (uint32_t)N * N;

    struct Ctx {
        T* S;
        uint32_t offF, offP, rowg;
        int rho, lane, z0, nz;
        int zb;                          // SLAB: stored plane of the run's z = 0
        uint32_t ey, eyp;               // edge warp: offsets in a plane of its staged row and of owned row lane + 1
        uint32_t exl, exr, exr1;        // the three edge columns
        const T *f0, *f1, *p0, *p1;
        T *of0, *of1, *op0, *op1;
        P dtcl2, dtcf2;
        SiteCoefs<T> K;
        P accg0, accg1, accvd, accvi;
    };

    static __device__ __forceinline__ bool edge_warp(const Ctx& C) { return C.rho == ROWS; }
    // array plane of run plane z0 + zrel: periodic in z for a whole lattice; a
    // slab's stored planes carry the halos, so no wrap
    static __device__ __forceinline__ uint32_t zplane(const Ctx& C, int zrel)
    {
        if constexpr (SLAB) return (uint32_t)(C.z0 + zrel + C.zb);
        else return (uint32_t)wrapn(C.z0 + zrel, N);
    }

    // plane z0 + zrel of the fields into slot `slot`: row warps their vectors,
    // the edge warp (lane r < ROWS for row r) the three edge scalars of each field
    template <int ROLE>
    static __device__ __forceinline__ void fetch_f(Ctx& C, int zrel, int slot)
    {
        const uint32_t zoff = zplane(C, zrel) * NN;
        if constexpr (ROLE != kEdge) {
            const uint32_t gi = zoff + C.rowg;
            T* d = C.S + slot * SLOTF + C.offF;
            cp_async16(d, C.f0 + gi);
            cp_async16(d + FIELDF, C.f1 + gi);
        } else if (C.lane < ROWS) {
            const uint32_t gb = zoff + C.ey;
            T* e = C.S + EF0 + slot * ESF + C.lane * 4;
            cp_async_small<sizeof(T)>(e + 0, C.f0 + gb + C.exl);
            cp_async_small<sizeof(T)>(e + 1, C.f0 + gb + C.exr);
            cp_async_small<sizeof(T)>(e + 2, C.f0 + gb + C.exr1);
            cp_async_small<sizeof(T)>(e + EF + 0, C.f1 + gb + C.exl);
            cp_async_small<sizeof(T)>(e + EF + 1, C.f1 + gb + C.exr);
            cp_async_small<sizeof(T)>(e + EF + 2, C.f1 + gb + C.exr1);
        }
    }
    // momenta of plane z0 + zrel: the computing rows' vectors, and the momenta at
    // x0 + W of the owned rows (edge warp, lane r - 1 for row r)
    template <int ROLE>
    static __device__ __forceinline__ void fetch_p(Ctx& C, int zrel, int slot)
    {
        const uint32_t zoff = zplane(C, zrel) * NN;
        if constexpr (ROLE != kEdge) {
            if constexpr (ROLE != kStage) {
                const uint32_t gi = zoff + C.rowg;
                T* d = C.S + P0 + slot * SLOTP + C.offP;
                cp_async16(d, C.p0 + gi);
                cp_async16(d + FIELDP, C.p1 + gi);
            }
        } else if (C.lane < TY) {
            const uint32_t gb = zoff + C.eyp + C.exr;
            T* e = C.S + EP0 + slot * ESP + C.lane;
            cp_async_small<sizeof(T)>(e, C.p0 + gb);
            cp_async_small<sizeof(T)>(e + EPF, C.p1 + gb);
        }
    }

    // ROLE (the same for the whole warp and the whole run): kOwn (rows 1..TY),
    // kAhead (the look-ahead row, computed but not stored), kStage (the halo
    // rows, staged only) or kEdge (the edge warp)
    template <int J, int ROLE>
    static __device__ __forceinline__ void plane(Ctx& C, int k)
    {
        const bool ahead = k == C.nz;
        constexpr bool edge = ROLE == kEdge;
        constexpr bool comp = ROLE == kOwn || ROLE == kAhead;
        constexpr bool own = ROLE == kOwn;
        cp_async_wait(D - 1);
        __syncthreads();
        if (k + D <= C.nz) {
            fetch_f<ROLE>(C, k + D + 1, (J + D + 2) % RF);
            fetch_p<ROLE>(C, k + D, (J + D) % RP);
        }
        cp_async_commit();
        if constexpr (ROLE == kStage) return;

        const T* Fm = C.S + (J % RF) * SLOTF;
        const T* Fc = C.S + ((J + 1) % RF) * SLOTF;
        const T* Fp = C.S + ((J + 2) % RF) * SLOTF;
        const T* Pc = C.S + P0 + (J % RP) * SLOTP;
        T* Gw = C.S + G0 + (J & 1) * SLOTP;
        const T* Gr = C.S + G0 + ((J + 1) & 1) * SLOTP;
        const T* Em = C.S + EF0 + (J % RF) * ESF;
        const T* Ec = C.S + EF0 + ((J + 1) % RF) * ESF;
        const T* Ep = C.S + EF0 + ((J + 2) % RF) * ESF;
        const T* Epc = C.S + EP0 + (J % RP) * ESP;
        T* EGw = C.S + EG0 + (J & 1) * 2 * TY;
        const T* EGr = C.S + EG0 + ((J + 1) & 1) * 2 * TY;

        if constexpr (edge) {
            // the boundary column x0 + W of owned row r = lane + 1, rounded as the
            // neighbouring tile rounds its own first column
            const int r = C.lane + 1;
            if (r <= TY && !ahead) {
                T c[2], pn[2];
#pragma unroll
                for (int f = 0; f < 2; f++) {
                    const T* e = Ec + f * EF;
                    const T cc = e[r * 4 + 1];
                    const T left = Fc[f * FIELDF + r * W + (W - 1)];
                    const T right = e[r * 4 + 2];
                    const T up = e[(r - 1) * 4 + 1], dn = e[(r + 1) * 4 + 1];
                    const T zm = Em[f * EF + r * 4 + 1], zp = Ep[f * EF + r * 4 + 1];
                    const T lap = s_add(s_add(s_add(s_sub(left, cc), s_sub(right, cc)), s_add(s_sub(up, cc), s_sub(dn, cc))),
                                        s_add(s_sub(zm, cc), s_sub(zp, cc)));
                    c[f] = cc;
                    pn[f] = s_fma(C.K.dtcl, lap, s_fma(C.K.dtcf, cc, Epc[f * EPF + (r - 1)]));
                }
                T g0, g1;
                site_kick_drift1<T>(C.K, c[0], c[1], pn[0], pn[1], g0, g1);
                EGw[r - 1] = g0;
                EGw[TY + (r - 1)] = g1;
            }
            return;
        }

        P cen[2][NP];
        T lefts[2], rights[2];
#pragma unroll
        for (int f = 0; f < 2; f++) {
            const T* Ff = Fc + f * FIELDF + C.offF;
            PK<T>::ld(Ff, cen[f]);
            // the tile's edge values: one broadcast load for the whole warp and a
            // select, no branch on the lane
            lefts[f] = ld_shared_if(C.lane == 0, Ec + f * EF + C.rho * 4 + 0,
                                    __shfl_up_sync(0xffffffffu, hi2(cen[f][NP - 1]), 1));
            rights[f] = ld_shared_if(C.lane == 31, Ec + f * EF + C.rho * 4 + 1,
                                     __shfl_down_sync(0xffffffffu, lo2(cen[f][0]), 1));
        }
        P g[2][NP];
        if (comp && !(ahead && ROLE == kAhead)) {
            P pn[2][NP];
#pragma unroll
            for (int f = 0; f < 2; f++) {
                const T* Ff = Fc + f * FIELDF + C.offF;
                P up[NP], dn[NP], zm[NP], zp[NP], pv[NP], lft[NP], rgt[NP];
                PK<T>::ld(Ff - W, up);
                PK<T>::ld(Ff + W, dn);
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
                    const uint32_t gi = zplane(C, k) * NN + C.rowg;
                    // the new state is read again only by the next step
                    PK<T>::st_stream(C.op0 + gi, pn[0]);
                    PK<T>::st_stream(C.op1 + gi, pn[1]);
                    PK<T>::st_stream(C.of0 + gi, g[0]);
                    PK<T>::st_stream(C.of1 + gi, g[1]);
                }
                PK<T>::st(Gw + C.offP, g[0]);
                PK<T>::st(Gw + FIELDP + C.offP, g[1]);
            }
        }
        // sums over the owned rows of plane k-1 (x and y pairs, potential) and
        // the z pair (k-1, k), from the new fields written one plane ago; lane
        // 31's x pair ends on the boundary column the edge warp computed
        if (k > 0 && own) {
            P gq[2][NP];
#pragma unroll
            for (int f = 0; f < 2; f++) {
                const T* Gf = Gr + f * FIELDP + C.offP;
                P yn[NP], xn[NP];
                PK<T>::ld(Gf, gq[f]);
                PK<T>::ld(Gf + W, yn);
                const T xnext = ld_shared_if(C.lane == 31, EGr + f * TY + (C.rho - 1),
                                             __shfl_down_sync(0xffffffffu, lo2(gq[f][0]), 1));
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
    template <int J, int ROLE>
    static __device__ __forceinline__ bool planes(Ctx& C, int k)
    {
        plane<J, ROLE>(C, k + J);
        if (k + J + 1 > C.nz) return false;
        if constexpr (J + 1 < PERIOD) return planes<J + 1, ROLE>(C, k);
        else return true;
    }
    // one run of planes: the prologue (planes z0 - 1 .. z0 + D of the fields,
    // z0 .. z0 + D - 1 of the momenta, one commit group per plane step), then the
    // planes; every role passes the same barriers
    template <int ROLE>
    static __device__ __forceinline__ void run(Ctx& C)
    {
        fetch_f<ROLE>(C, -1, 0);
        fetch_f<ROLE>(C, 0, 1);
        fetch_f<ROLE>(C, 1, 2);
        fetch_p<ROLE>(C, 0, 0);
        cp_async_commit();
#pragma unroll
        for (int j = 1; j < D; j++) {
            fetch_f<ROLE>(C, j + 1, j + 2);
            fetch_p<ROLE>(C, j, j);
            cp_async_commit();
        }
        for (int k = 0; planes<0, ROLE>(C, k); k += PERIOD) {}
    }
};

template <typename T, int N, int TY, int D, bool SLAB>
__global__ void __launch_bounds__(XW<T, N, TY, D, SLAB>::THREADS, 1)
    step_xw_kernel(Bufs<T> B, Model M, DevScalars* sc, double* partials, SlabRun R)
{
    typedef XW<T, N, TY, D, SLAB> F;
    constexpr int VW = F::VW, W = F::W, NXT = F::NXT;
    __shared__ double red[32 * kSums];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (sc->status != LAT_OK) return;

    typename F::Ctx C;
    C.S = reinterpret_cast<T*>(smem_raw);
    C.rho = threadIdx.x >> 5;                      // the warp's staged row, or ROWS for the edge warp
    C.lane = threadIdx.x & 31;
    C.offF = (uint32_t)C.rho * W + C.lane * VW;
    C.offP = (uint32_t)(C.rho >= 1 && C.rho <= TY + 1 ? C.rho - 1 : 0) * W + C.lane * VW;
    const bool par = (sc->step & 1) != 0;
    if constexpr (!SLAB) {
        C.f0 = par ? B.f[1][0] : B.f[0][0];
        C.f1 = par ? B.f[1][1] : B.f[0][1];
        C.p0 = par ? B.p[1][0] : B.p[0][0];
        C.p1 = par ? B.p[1][1] : B.p[0][1];
        C.of0 = par ? B.f[0][0] : B.f[1][0];
        C.of1 = par ? B.f[0][1] : B.f[1][1];
        C.op0 = par ? B.p[0][0] : B.p[1][0];
        C.op1 = par ? B.p[0][1] : B.p[1][1];
    }
    C.K = site_coefs<T>(sc, M.beta);
    C.dtcl2 = mk2(C.K.dtcl, C.K.dtcl);
    C.dtcf2 = mk2(C.K.dtcf, C.K.dtcf);
    C.accg0 = C.accg1 = C.accvd = C.accvi = mk2(T(0), T(0));

    // groups of NXT blocks: the x tiles of one y tile, marching the same
    // (y tile, z plane) units
    const int ngroups = gridDim.x / NXT;
    const int grp = blockIdx.x / NXT, xt = blockIdx.x - grp * NXT;
    const Layout Lw = tile_layout(N / TY, ngroups, grp, SLAB ? R.nz : N);
    const int x0 = xt * W;
    // edge columns (periodic in x)
    C.exl = (uint32_t)(x0 == 0 ? N - 1 : x0 - 1);
    C.exr = (uint32_t)(x0 + W == N ? 0 : x0 + W);
    C.exr1 = (uint32_t)(x0 + W + 1 >= N ? x0 + W + 1 - N : x0 + W + 1);
    C.zb = 0;
    int u = Lw.ubeg;
    for (bool first = true; u < Lw.uend; first = false) {
        const int zt = Lw.zspan;   // planes per y tile in this group's unit space
        const int yt = u / zt;
        const int zrel = u - yt * zt;
        C.z0 = Lw.zoff + zrel;
        C.nz = min(zt - zrel, Lw.uend - u);
        if constexpr (SLAB) {
            // the range holding plane z0 of the end-to-end z space: the run stays
            // within it, on its slab's arrays, from its stored planes
            int r = 0;
            while (r + 1 < R.nranges && C.z0 >= R.rz[r + 1]) r++;
            C.z0 -= R.rz[r];
            C.nz = min(C.nz, R.rn[r] - C.z0);
            C.zb = R.rzb[r];
            void* const* bs = R.buf[R.rslab[r]];
            C.f0 = (const T*)bs[par ? 4 : 0];
            C.f1 = (const T*)bs[par ? 5 : 1];
            C.p0 = (const T*)bs[par ? 6 : 2];
            C.p1 = (const T*)bs[par ? 7 : 3];
            C.of0 = (T*)bs[par ? 0 : 4];
            C.of1 = (T*)bs[par ? 1 : 5];
            C.op0 = (T*)bs[par ? 2 : 6];
            C.op1 = (T*)bs[par ? 3 : 7];
        }
        u += C.nz;
        const int rrow = F::edge_warp(C) ? C.lane : C.rho;   // the row this thread stages
        C.rowg = (uint32_t)wrapn(yt * TY - 1 + (F::edge_warp(C) ? 0 : C.rho), N) * N + x0 + C.lane * VW;
        C.ey = (uint32_t)wrapn(yt * TY - 1 + min(rrow, F::ROWS - 1), N) * N;
        C.eyp = (uint32_t)wrapn(yt * TY + min(C.lane, TY - 1), N) * N;
        // the previous segment's last plane is read by every thread before the
        // prologue refills the ring
        if (!first) __syncthreads();
        if (F::edge_warp(C)) F::template run<kEdge>(C);
        else if (C.rho == 0 || C.rho == F::ROWS - 1) F::template run<kStage>(C);
        else if (C.rho == TY + 1) F::template run<kAhead>(C);
        else F::template run<kOwn>(C);
    }

    T v[kSums] = {lo2(C.accg0) + hi2(C.accg0), lo2(C.accg1) + hi2(C.accg1),
                  (lo2(C.accvd) + hi2(C.accvd)) * site_vsum_factor<T>(C.K.quartic),
                  T(0.5) * (lo2(C.accvi) + hi2(C.accvi))};
    if constexpr (SLAB) finish_block_sums(M, sc, partials, v, red, R.sums_out);
    else finish_block(M, sc, partials, v, red, true);
}

} // namespace xw

} // namespace lat
