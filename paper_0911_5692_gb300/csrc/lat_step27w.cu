// lat_step27w.cu -- the fused leapfrog step with the 27-point Laplacian of
// Sec. II.C (Patra and Karttunen) over x tiles one warp wide, with the lattice
// side N, the tile height TY and the prefetch depth D known at compile time
// (variant 5 of the 27-point stencil).
//
// Tiles, ring and edge warp follow the 7-point kernel of lat_step_xw.cu: a tile
// is W = 32 16-byte vectors wide and TY rows tall, warp r stages row r (0: the
// halo row below, 1..TY: the owned rows, TY + 1: the look-ahead row, TY + 2: the
// halo row above), and one more warp (the edge warp) stages the scalars of the
// tile's x neighbours, columns x0 - 1, x0 + W and x0 + W + 1, and computes the
// new fields of the boundary column x0 + W, rounded exactly as the next tile
// computes its own first column.
//
// Laplacian. In units of 1/(30 dx^2) the weights are 14 (6 faces), 3 (12 edges)
// and 1 (8 corners). Per plane p and site, with differences taken from that
// plane's own centre C:
//   v = (f(y - 1) - C) + (f(y + 1) - C)                the y pair
//   h = (f(x + 1) - C) - (C - f(x - 1))                the x pair
//   e = h + v                                          the 4 in-plane faces
//   k = v(x - 1) + v(x + 1) + 2 h                      the 4 in-plane corners
// (v(x +- 1) is taken about C(x +- 1); 2 h puts back the 2 (C(x +- 1) - C)),
//   q_p = 3 e + k    the plane's part when it is the plane below or above,
//   r_p = 14 e + 3 k its part when it is the centre plane, and
//   30 dx^2 Lap f(z) = r_z + q_{z-1} + q_{z+1} + 30 ((C_{z-1} - C_z) + (C_{z+1} - C_z)).
// Every term is a sum of differences of neighbouring values (exact for
// f = const + small). The x-shifted sums are formed by scalar operations that
// write the halves of the packed pairs, so no register moves build shifted
// pairs. Along z each field keeps two packed values per site in registers:
// the pending sum of plane z, L_z = (q_{z-1} - 30 (C_z - C_{z-1})) + r_z, and
// q_z (C_z is read again from the ring); plane z + 1's aggregate, formed once,
// completes
// Lap(z) = (L_z + 30 (C_{z+1} - C_z)) + q_{z+1} and starts L_{z+1}. Every site's
// value depends only on its 3x3x3 neighbourhood, not on the tiling or the z
// segments.
//
// Sums of the new fields for eq. scale: -<g Lap g> is the mean over sites of
// sum_b w_b (g(x + b) - g(x))^2 over the 13 bonds a site owns (all with
// dy >= 0; the three with dz = -1 counted from the site above, as bonds between
// rows y (plane P + 1) and y + 1 (plane P)). Each bond is summed by the warp of
// its lower row at the column of its left end, so the only x neighbour a lane
// needs is on its right: the next lane's first site, or for lane 31 the
// boundary column. Bonds between planes P and P + 1 are summed at plane P + 2
// from a ring of new-field planes, after the barrier that completes both.
//
// The NXT = N / W x tiles of a y tile are taken by NXT consecutive blocks that
// march the same (y tile, z plane) units, so the edge scalars lie in memory
// lines the neighbouring blocks are reading too (L2 hits).
#include <algorithm>

#include "lat_async.cuh"
#include "lat_kernels.h"
#include "lat_pairs.cuh"
#include "lat_site.cuh"

namespace lat {

namespace {

constexpr unsigned kFull = 0xffffffffu;
enum { kOwn, kAhead, kStage, kEdge };   // warp roles

template <int D>
struct Ring27W {
    static constexpr int RF = D == 1 ? 4 : 6;          // field plane slots (>= D + 3)
    static constexpr int RP = D + 1;                   // momentum plane slots
    static constexpr int GS = D == 1 ? 4 : 3;          // new-field plane slots (3 in use)
    static constexpr int PERIOD = D == 1 ? 4 : 6;      // lcm(RF, RP, GS)
    static_assert(RF >= D + 3 && GS >= 3 && PERIOD % RF == 0 && PERIOD % RP == 0 && PERIOD % GS == 0,
                  "ring period");
};

template <typename T, int N, int TY, int D>
struct S27 {
    typedef typename PK<T>::P P;
    static constexpr int RF = Ring27W<D>::RF, RP = Ring27W<D>::RP, GS = Ring27W<D>::GS;
    static constexpr int PERIOD = Ring27W<D>::PERIOD;
    static constexpr int NP = PK<T>::NP;
    static constexpr int VW = 2 * NP;                  // elements per 16-byte vector
    static constexpr int W = 32 * VW;                  // tile width: one warp of vectors
    static constexpr int NXT = N / W;                  // x tiles per row
    static constexpr int ROWS = TY + 3;                // staged rows (one warp each)
    static constexpr int GR = TY + 1;                  // computed rows (owned + look-ahead)
    static constexpr int THREADS = (ROWS + 1) * 32;    // and the edge warp
    static_assert(N % W == 0 && N % TY == 0 && GR <= 32, "tile geometry");
    // Shared memory, in elements. The field ring [slot][field][ROWS][RS] with a
    // row stride one vector longer than the tile (the edge warp reads the last
    // column of every row: the padding spreads those reads over the banks), the
    // momentum ring [slot][field][GR][W], the new-field ring [slot][field][GR][W];
    // then the edge scalars: fields [slot][field][ROWS][4] (x0 - 1, x0 + W,
    // x0 + W + 1, unused), momenta at x0 + W [slot][field][GR], new fields at
    // x0 + W [slot][field][GR].
    static constexpr int RS = W + VW;
    static constexpr uint32_t FIELDF = ROWS * RS, SLOTF = 2 * FIELDF;
    static constexpr uint32_t FIELDP = GR * W, SLOTP = 2 * FIELDP;
    static constexpr uint32_t P0 = RF * SLOTF, G0 = P0 + RP * SLOTP;
    static constexpr uint32_t EF = ROWS * 4, ESF = 2 * EF;
    static constexpr uint32_t ESP = 2 * GR;
    static constexpr uint32_t EF0 = G0 + GS * SLOTP, EP0 = EF0 + RF * ESF, EG0 = EP0 + RP * ESP;
    static constexpr uint32_t END = EG0 + GS * ESP;
    static constexpr size_t SMEM = (sizeof(T) * (size_t)END + 15) / 16 * 16;
    static constexpr uint32_t NN = (uint32_t)N * N;

    struct Ctx {
        T* S;
        uint32_t offF, offP, rowg;
        int rho, lane, z0, nz;
        uint32_t ey, eyp;               // edge warp: the row of its staged lane and of computed row lane + 1
        uint32_t exl, exr, exr1;        // the three edge columns
        const T *f0, *f1, *p0, *p1;
        T *of0, *of1, *op0, *op1;
        SiteCoefs<T> K;
        P Lz[2][NP], Qz[2][NP];              // per field: L_z and q_z (row warps)
        T eL[2], eQ[2], eC[2];               // L_z, q_z and C_z at the boundary column (edge warp)
        P wg[2], vd, vi;                     // sums of the new fields
    };

    static __device__ __forceinline__ bool edge_warp(const Ctx& C) { return C.rho == ROWS; }

    // plane z0 + zrel of the fields into ring slot `slot`
    template <int ROLE>
    static __device__ __forceinline__ void fetch_f(Ctx& C, int zrel, int slot)
    {
        const uint32_t zoff = (uint32_t)wrapn(C.z0 + zrel, N) * NN;
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
    // momenta of plane z0 + zrel for the computed rows, and at x0 + W (edge warp,
    // lane r - 1 for row r)
    template <int ROLE>
    static __device__ __forceinline__ void fetch_p(Ctx& C, int zrel, int slot)
    {
        const uint32_t zoff = (uint32_t)wrapn(C.z0 + zrel, N) * NN;
        if constexpr (ROLE != kEdge) {
            if constexpr (ROLE != kStage) {
                const uint32_t gi = zoff + C.rowg;
                T* d = C.S + P0 + slot * SLOTP + C.offP;
                cp_async16(d, C.p0 + gi);
                cp_async16(d + FIELDP, C.p1 + gi);
            }
        } else if (C.lane < GR) {
            const uint32_t gb = zoff + C.eyp + C.exr;
            T* e = C.S + EP0 + slot * ESP + C.lane;
            cp_async_small<sizeof(T)>(e, C.p0 + gb);
            cp_async_small<sizeof(T)>(e + GR, C.p1 + gb);
        }
    }

    // x neighbours of this lane's vector: from the adjacent lanes, at the tile's
    // ends the edge scalars (*el at x0 - 1, *er at x0 + W), read by those lanes
    // only. Every lane calls this.
    static __device__ __forceinline__ void xnb(const P (&v)[NP], const T* el, const T* er, int lane, T& l, T& r)
    {
        l = ld_shared_if(lane == 0, el, __shfl_up_sync(kFull, hi2(v[NP - 1]), 1));
        r = ld_shared_if(lane == 31, er, __shfl_down_sync(kFull, lo2(v[0]), 1));
    }

    // The aggregates of one field at this lane's sites of row rho: centres c,
    // q = 3 e + k and r = 14 e + 3 k. F: the field's plane in the ring, E: its
    // edge scalars. Every lane calls this.
    static __device__ __forceinline__ void aggr(const Ctx& C, const T* F, const T* E, P (&c)[NP], P (&q)[NP],
                                                P (&r)[NP])
    {
        const T* row = F + C.offF;
        P m[NP], p[NP];
        PK<T>::ld(row, c);
        PK<T>::ld(row - RS, m);
        PK<T>::ld(row + RS, p);
        const T* e = E + C.rho * 4;
        T cl, cr, ml, mr, pl, pr;
        xnb(c, e, e + 1, C.lane, cl, cr);
        xnb(m, e - 4, e - 3, C.lane, ml, mr);
        xnb(p, e + 4, e + 5, C.lane, pl, pr);
        P v[NP];
        T cs[VW + 2], vs[VW + 2];
#pragma unroll
        for (int j = 0; j < NP; j++) {
            v[j] = add2(sub2(m[j], c[j]), sub2(p[j], c[j]));
            cs[1 + 2 * j] = lo2(c[j]);
            cs[2 + 2 * j] = hi2(c[j]);
            vs[1 + 2 * j] = lo2(v[j]);
            vs[2 + 2 * j] = hi2(v[j]);
        }
        cs[0] = cl;
        cs[VW + 1] = cr;
        vs[0] = s_add(s_sub(ml, cl), s_sub(pl, cl));
        vs[VW + 1] = s_add(s_sub(mr, cr), s_sub(pr, cr));
        T dd[VW + 1];   // differences of consecutive sites
#pragma unroll
        for (int i = 0; i <= VW; i++) dd[i] = s_sub(cs[i + 1], cs[i]);
        const P two = mk2(T(2), T(2)), three = mk2(T(3), T(3)), fourteen = mk2(T(14), T(14));
#pragma unroll
        for (int j = 0; j < NP; j++) {
            const int a = 1 + 2 * j, b = 2 + 2 * j;   // positions of the pair's sites in cs and vs
            const P h = mk2(s_sub(dd[a], dd[a - 1]), s_sub(dd[b], dd[b - 1]));
            const P t = mk2(s_add(vs[a - 1], vs[a + 1]), s_add(vs[b - 1], vs[b + 1]));
            const P k = fma2(two, h, t);
            const P eh = add2(h, v[j]);
            q[j] = fma2(three, eh, k);
            r[j] = fma2(fourteen, eh, mul2(three, k));
        }
    }

    // The same aggregates at one site, rounded as the first site of a vector:
    // the centre row at x - 1, x, x + 1 (cl, c0, c1) and the rows y - 1 (m*) and
    // y + 1 (p*) at the same columns.
    static __device__ __forceinline__ void aggr1(T cl, T c0, T c1, T ml, T m0, T m1, T pl, T p0, T p1, T& q, T& r)
    {
        const T vl = s_add(s_sub(ml, cl), s_sub(pl, cl));
        const T v0 = s_add(s_sub(m0, c0), s_sub(p0, c0));
        const T v1 = s_add(s_sub(m1, c1), s_sub(p1, c1));
        const T h = s_sub(s_sub(c1, c0), s_sub(c0, cl));
        const T k = s_fma(T(2), h, s_add(vl, v1));
        const T eh = s_add(h, v0);
        q = s_fma(T(3), eh, k);
        r = s_fma(T(14), eh, s_mul(T(3), k));
    }

    // Edge warp: the aggregates at (x0 + W, row r) of one field's plane F (ring)
    // with edge scalars E; the site's centre in *c.
    static __device__ __forceinline__ void aggr_edge(const T* F, const T* E, int r, T& c, T& q, T& r_)
    {
        const T* lc = F + r * RS + (W - 1);
        const T* e = E + r * 4;
        c = e[1];
        aggr1(lc[0], e[1], e[2], lc[-RS], e[-3], e[-2], lc[RS], e[5], e[6], q, r_);
    }

    // Bonds of the new-field planes P (Gp) and P + 1 (Gu) at this lane's sites
    // of owned row rho, and the potential sums of plane P. EGp, EGu: the
    // boundary column of both planes. Every lane of an owned row calls this.
    static __device__ __forceinline__ void bonds(Ctx& C, const T* Gp, const T* Gu, const T* EGp, const T* EGu)
    {
        P pz[2][NP];
#pragma unroll
        for (int f = 0; f < 2; f++) {
            const T* gp = Gp + f * FIELDP + C.offP;
            const T* gu = Gu + f * FIELDP + C.offP;
            P p0[NP], p1[NP], u0[NP], u1[NP];
            PK<T>::ld(gp, p0);
            PK<T>::ld(gp + W, p1);
            PK<T>::ld(gu, u0);
            PK<T>::ld(gu + W, u1);
            const int eb = f * GR + C.rho - 1;
            // right neighbours of element VW - 1; lane 31: the boundary column
            const bool last = C.lane == 31;
            const T p0e = ld_shared_if(last, EGp + eb, __shfl_down_sync(kFull, lo2(p0[0]), 1));
            const T p1e = ld_shared_if(last, EGp + eb + 1, __shfl_down_sync(kFull, lo2(p1[0]), 1));
            const T u0e = ld_shared_if(last, EGu + eb, __shfl_down_sync(kFull, lo2(u0[0]), 1));
            const T u1e = ld_shared_if(last, EGu + eb + 1, __shfl_down_sync(kFull, lo2(u1[0]), 1));
            // the rows shifted one site to the right
            P p0R[NP], p1R[NP], u0R[NP], u1R[NP];
#pragma unroll
            for (int j = 0; j < NP; j++) {
                const bool lastj = j == NP - 1;
                p0R[j] = mk2(hi2(p0[j]), lastj ? p0e : lo2(p0[lastj ? j : j + 1]));
                p1R[j] = mk2(hi2(p1[j]), lastj ? p1e : lo2(p1[lastj ? j : j + 1]));
                u0R[j] = mk2(hi2(u0[j]), lastj ? u0e : lo2(u0[lastj ? j : j + 1]));
                u1R[j] = mk2(hi2(u1[j]), lastj ? u1e : lo2(u1[lastj ? j : j + 1]));
            }
            const P zero = mk2(T(0), T(0));
            P a14 = zero, a3 = zero, a1 = zero;
#pragma unroll
            for (int j = 0; j < NP; j++) {
                const P c = p0[j];
                P d;
                // faces: (1,0,0) (0,1,0) (0,0,1)
                d = sub2(p0R[j], c); a14 = fma2(d, d, a14);
                d = sub2(p1[j], c);  a14 = fma2(d, d, a14);
                d = sub2(u0[j], c);  a14 = fma2(d, d, a14);
                // edges: (1,1,0) (-1,1,0) (1,0,1) (-1,0,1) (0,1,1), and (0,1,-1) from the site above
                d = sub2(p1R[j], c);      a3 = fma2(d, d, a3);
                d = sub2(p1[j], p0R[j]);  a3 = fma2(d, d, a3);
                d = sub2(u0R[j], c);      a3 = fma2(d, d, a3);
                d = sub2(u0[j], p0R[j]);  a3 = fma2(d, d, a3);
                d = sub2(u1[j], c);       a3 = fma2(d, d, a3);
                d = sub2(p1[j], u0[j]);   a3 = fma2(d, d, a3);
                // corners: (1,1,1) (-1,1,1), and (1,1,-1) (-1,1,-1) from the site above
                d = sub2(u1R[j], c);      a1 = fma2(d, d, a1);
                d = sub2(u1[j], p0R[j]);  a1 = fma2(d, d, a1);
                d = sub2(p1R[j], u0[j]);  a1 = fma2(d, d, a1);
                d = sub2(p1[j], u0R[j]);  a1 = fma2(d, d, a1);
                pz[f][j] = c;
            }
            // this plane's bonds by weight, folded into the field's sum
            C.wg[f] = fma2(mk2(T(14), T(14)), a14, fma2(mk2(T(3), T(3)), a3, add2(a1, C.wg[f])));
        }
#pragma unroll
        for (int j = 0; j < NP; j++) site_vsum<T>(C.K, pz[0][j], pz[1][j], C.vd, C.vi);
    }

    // the top of every plane: wait for plane k + 1 (and its momenta), the
    // barrier, then the prefetch of plane k + D + 1
    template <int J, int ROLE>
    static __device__ __forceinline__ void plane_top(Ctx& C, int k)
    {
        cp_async_wait(D - 1);
        __syncthreads();
        if (k + D <= C.nz) {
            fetch_f<ROLE>(C, k + D + 1, (J + D + 2) % RF);
            fetch_p<ROLE>(C, k + D, (J + D) % RP);
        }
        cp_async_commit();
    }
    // the prologue of a run: planes z0 - 1 .. z0 + D of the fields, z0 .. z0 + D - 1
    // of the momenta, one commit group per plane step
    template <int ROLE>
    static __device__ __forceinline__ void prologue(Ctx& C)
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
    }

    // Edge warp, plane k: the boundary column x0 + W of computed row r = lane + 1.
    template <int J>
    static __device__ __forceinline__ void plane_edge(Ctx& C, int k)
    {
        plane_top<J, kEdge>(C, k);
        const int r = C.lane + 1;
        if (r > GR) return;
        const T* Fm = C.S + (J % RF) * SLOTF;
        const T* Fc = C.S + ((J + 1) % RF) * SLOTF;
        const T* Fp = C.S + ((J + 2) % RF) * SLOTF;
        const T* Em = C.S + EF0 + (J % RF) * ESF;
        const T* Ec = C.S + EF0 + ((J + 1) % RF) * ESF;
        const T* Ep = C.S + EF0 + ((J + 2) % RF) * ESF;
        const T* Epc = C.S + EP0 + (J % RP) * ESP;
        T* EGw = C.S + EG0 + (J % GS) * ESP;
        if (J == 0 && k == 0) {   // the first plane of a run: L and q of planes z0 - 1 and z0
#pragma unroll
            for (int f = 0; f < 2; f++) {
                T cm, qm, rm, cc, qc, rc;
                aggr_edge(Fm + f * FIELDF, Em + f * EF, r, cm, qm, rm);
                aggr_edge(Fc + f * FIELDF, Ec + f * EF, r, cc, qc, rc);
                C.eL[f] = s_add(s_fma(T(-30), s_sub(cc, cm), qm), rc);
                C.eQ[f] = qc;
                C.eC[f] = cc;
            }
        }
        T cz[2], pn[2];
#pragma unroll
        for (int f = 0; f < 2; f++) {
            T cp, qp, rp;
            aggr_edge(Fp + f * FIELDF, Ep + f * EF, r, cp, qp, rp);
            const T d = s_sub(cp, C.eC[f]);
            const T lap = s_add(s_fma(T(30), d, C.eL[f]), qp);
            pn[f] = s_fma(C.K.dtcl, lap, s_fma(C.K.dtcf, C.eC[f], Epc[f * GR + (r - 1)]));
            C.eL[f] = s_add(s_fma(T(-30), d, C.eQ[f]), rp);
            C.eQ[f] = qp;
            cz[f] = C.eC[f];
            C.eC[f] = cp;
        }
        T g0, g1;
        site_kick_drift1<T>(C.K, cz[0], cz[1], pn[0], pn[1], g0, g1);
        EGw[r - 1] = g0;
        EGw[GR + (r - 1)] = g1;
    }

    // Row warps, plane k: kick and drift of the computed rows, and the bonds of
    // planes k - 2 and k - 1 (both written before the barrier) for the owned rows.
    // ROLE (the same for the whole warp and the whole run): kOwn, kAhead (the
    // look-ahead row, computed but not stored) or kStage (the halo rows, staged
    // only).
    template <int J, int ROLE>
    static __device__ __forceinline__ void plane_rows(Ctx& C, int k)
    {
        plane_top<J, ROLE>(C, k);
        constexpr bool comp = ROLE != kStage;
        constexpr bool own = ROLE == kOwn;
        const T* Fm = C.S + (J % RF) * SLOTF;
        const T* Fc = C.S + ((J + 1) % RF) * SLOTF;
        const T* Fp = C.S + ((J + 2) % RF) * SLOTF;
        const T* Pc = C.S + P0 + (J % RP) * SLOTP;
        T* Gw = C.S + G0 + (J % GS) * SLOTP;
        const T* Gm1 = C.S + G0 + ((J + GS - 1) % GS) * SLOTP;   // plane k - 1
        const T* Gm2 = C.S + G0 + ((J + GS - 2) % GS) * SLOTP;   // plane k - 2
        const T* Em = C.S + EF0 + (J % RF) * ESF;
        const T* Ec = C.S + EF0 + ((J + 1) % RF) * ESF;
        const T* Ep = C.S + EF0 + ((J + 2) % RF) * ESF;
        const T* EGm1 = C.S + EG0 + ((J + GS - 1) % GS) * ESP;
        const T* EGm2 = C.S + EG0 + ((J + GS - 2) % GS) * ESP;

        if (comp) {
            const P c30 = mk2(T(30), T(30)), cm30 = mk2(T(-30), T(-30));
            if (J == 0 && k == 0) {   // the first plane of a run: L and q of planes z0 - 1 and z0
#pragma unroll
                for (int f = 0; f < 2; f++) {
                    P cm[NP], qm[NP], rm[NP], cc[NP], qc[NP], rc[NP];
                    aggr(C, Fm + f * FIELDF, Em + f * EF, cm, qm, rm);
                    aggr(C, Fc + f * FIELDF, Ec + f * EF, cc, qc, rc);
#pragma unroll
                    for (int j = 0; j < NP; j++) {
                        C.Lz[f][j] = add2(fma2(cm30, sub2(cc[j], cm[j]), qm[j]), rc[j]);
                        C.Qz[f][j] = qc[j];
                    }
                }
            }
            P pn[2][NP], cz[2][NP];
            const P dtcl2 = mk2(C.K.dtcl, C.K.dtcl), dtcf2 = mk2(C.K.dtcf, C.K.dtcf);
#pragma unroll
            for (int f = 0; f < 2; f++) {
                P cp[NP], qp[NP], rp[NP], pv[NP];
                PK<T>::ld(Fc + f * FIELDF + C.offF, cz[f]);   // C_z
                aggr(C, Fp + f * FIELDF, Ep + f * EF, cp, qp, rp);
                PK<T>::ld(Pc + f * FIELDP + C.offP, pv);
#pragma unroll
                for (int j = 0; j < NP; j++) {
                    const P d = sub2(cp[j], cz[f][j]);
                    const P lap = add2(fma2(c30, d, C.Lz[f][j]), qp[j]);
                    pn[f][j] = fma2(dtcl2, lap, fma2(dtcf2, cz[f][j], pv[j]));
                    C.Lz[f][j] = add2(fma2(cm30, d, C.Qz[f][j]), rp[j]);
                    C.Qz[f][j] = qp[j];
                }
            }
            P g[2][NP];
            // potential part of the kick and the drift (lat_site.cuh)
#pragma unroll
            for (int j = 0; j < NP; j++) site_kick_drift<T>(C.K, cz[0][j], cz[1][j], pn[0][j], pn[1][j], g[0][j], g[1][j]);
            if (own && k < C.nz) {
                const uint32_t gi = (uint32_t)(C.z0 + k) * NN + C.rowg;
                PK<T>::st(C.op0 + gi, pn[0]);
                PK<T>::st(C.op1 + gi, pn[1]);
                PK<T>::st(C.of0 + gi, g[0]);
                PK<T>::st(C.of1 + gi, g[1]);
            }
            PK<T>::st(Gw + C.offP, g[0]);
            PK<T>::st(Gw + FIELDP + C.offP, g[1]);
        }
        if (own && k >= 2) bonds(C, Gm2, Gm1, EGm2, EGm1);
    }

    // planes k + J .. k + PERIOD - 1; false once the look-ahead plane is done
    template <int J, int ROLE>
    static __device__ __forceinline__ bool planes(Ctx& C, int k)
    {
        if constexpr (ROLE == kEdge) plane_edge<J>(C, k + J);
        else plane_rows<J, ROLE>(C, k + J);
        if (k + J + 1 > C.nz) return false;
        if constexpr (J + 1 < PERIOD) return planes<J + 1, ROLE>(C, k);
        else return true;
    }
    template <int ROLE>
    static __device__ __forceinline__ void run(Ctx& C)
    {
        prologue<ROLE>(C);
        for (int k = 0; planes<0, ROLE>(C, k); k += PERIOD) {}
    }
};

template <typename T, int N, int TY, int D>
__global__ void __launch_bounds__(S27<T, N, TY, D>::THREADS, 1)
    step27w_kernel(Bufs<T> B, Model M, DevScalars* sc, double* partials)
{
    typedef S27<T, N, TY, D> F;
    constexpr int VW = F::VW, W = F::W, NXT = F::NXT;
    __shared__ double red[32 * kSums];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (sc->status != LAT_OK) return;

    typename F::Ctx C;
    C.S = reinterpret_cast<T*>(smem_raw);
    C.rho = threadIdx.x >> 5;                      // the warp's staged row, or ROWS for the edge warp
    C.lane = threadIdx.x & 31;
    C.offF = (uint32_t)C.rho * F::RS + C.lane * VW;
    C.offP = (uint32_t)(C.rho >= 1 && C.rho <= F::GR ? C.rho - 1 : 0) * W + C.lane * VW;
    const bool par = (sc->step & 1) != 0;
    C.f0 = par ? B.f[1][0] : B.f[0][0];
    C.f1 = par ? B.f[1][1] : B.f[0][1];
    C.p0 = par ? B.p[1][0] : B.p[0][0];
    C.p1 = par ? B.p[1][1] : B.p[0][1];
    C.of0 = par ? B.f[0][0] : B.f[1][0];
    C.of1 = par ? B.f[0][1] : B.f[1][1];
    C.op0 = par ? B.p[0][0] : B.p[1][0];
    C.op1 = par ? B.p[0][1] : B.p[1][1];
    C.K = site_coefs<T>(sc, M.beta);
    const typename F::P zero = mk2(T(0), T(0));
    C.wg[0] = C.wg[1] = C.vd = C.vi = zero;

    // groups of NXT blocks: the x tiles of one y tile, marching the same
    // (y tile, z plane) units (an equal share of the (N / TY) * N units per group)
    const int ngroups = gridDim.x / NXT;
    const int grp = blockIdx.x / NXT, xt = blockIdx.x - grp * NXT;
    const int x0 = xt * W;
    C.exl = (uint32_t)(x0 == 0 ? N - 1 : x0 - 1);
    C.exr = (uint32_t)(x0 + W == N ? 0 : x0 + W);
    C.exr1 = (uint32_t)(x0 + W + 1 >= N ? x0 + W + 1 - N : x0 + W + 1);
    constexpr long long U = (long long)(N / TY) * N;
    long long u = (long long)grp * U / ngroups;
    const long long uend = ((long long)grp + 1) * U / ngroups;
    for (bool first = true; u < uend; first = false) {
        const int yt = (int)(u / N);
        C.z0 = (int)(u - (long long)yt * N);
        C.nz = (int)min((long long)(N - C.z0), uend - u);
        u += C.nz;
        C.rowg = (uint32_t)wrapn(yt * TY - 1 + (F::edge_warp(C) ? 0 : C.rho), N) * N + x0 + C.lane * VW;
        C.ey = (uint32_t)wrapn(yt * TY - 1 + min(C.lane, F::ROWS - 1), N) * N;
        C.eyp = (uint32_t)wrapn(yt * TY + min(C.lane, F::GR - 1), N) * N;
        // every thread is done with the previous segment's ring before the
        // prologue refills it
        if (!first) __syncthreads();
        // the same barriers on every path: one per plane, one after the run
        if (F::edge_warp(C)) F::template run<kEdge>(C);
        else if (C.rho == 0 || C.rho == F::ROWS - 1) F::template run<kStage>(C);
        else if (C.rho == F::GR) F::template run<kAhead>(C);
        else F::template run<kOwn>(C);
        // the last bonds: planes nz - 1 and nz (the look-ahead plane)
        __syncthreads();
        if (!F::edge_warp(C) && C.rho >= 1 && C.rho <= TY) {
            const int gb = (C.nz - 1) % F::GS, gl = C.nz % F::GS;
            F::bonds(C, C.S + F::G0 + gb * F::SLOTP, C.S + F::G0 + gl * F::SLOTP, C.S + F::EG0 + gb * F::ESP,
                     C.S + F::EG0 + gl * F::ESP);
        }
    }

    double v[kSums];
    for (int f = 0; f < 2; f++) v[f] = (double)lo2(C.wg[f]) + (double)hi2(C.wg[f]);
    v[2] = ((double)lo2(C.vd) + (double)hi2(C.vd)) * (double)site_vsum_factor<T>(C.K.quartic);
    v[3] = 0.5 * ((double)lo2(C.vi) + (double)hi2(C.vi));
    finish_block(M, sc, partials, v, red, true);
}

// Compiled instances: (element bytes, N, TY, D).
struct Key27W {
    int esize, n, ty, depth;
};
constexpr Key27W k27W[] = {{4, 256, 16, 1}, {4, 512, 16, 1}, {8, 256, 16, 1}, {8, 512, 16, 1}};

template <typename T>
const void* s27w_fn(int n, int ty, int depth, size_t* smem)
{
#define LAT_S27W_CASE(NN, TT, DD)                                \
    if (n == NN && ty == TT && depth == DD) {                    \
        *smem = S27<T, NN, TT, DD>::SMEM;                        \
        return (const void*)step27w_kernel<T, NN, TT, DD>;       \
    }
    LAT_S27W_CASE(256, 16, 1) LAT_S27W_CASE(512, 16, 1)
#undef LAT_S27W_CASE
    return nullptr;
}

const void* s27w_kernel(int esize, int n, int ty, int depth, size_t* smem)
{
    for (const Key27W& k : k27W)
        if (k.esize == esize && k.n == n && k.ty == ty && k.depth == depth)
            return esize == 4 ? s27w_fn<float>(n, ty, depth, smem) : s27w_fn<double>(n, ty, depth, smem);
    return nullptr;
}

} // namespace

bool s27w_config(int n, int elem_bytes, int ty, int zr, int depth, MarchConfig* cfg)
{
    const int tyv = ty > 0 ? ty : 16;
    const int d = depth > 0 ? depth : 1;
    size_t smem = 0;
    const void* fn = s27w_kernel(elem_bytes, n, tyv, d, &smem);
    if (!fn || smem > 227 * 1024 - 2048) return false;
    const int vw = 16 / elem_bytes, w = 32 * vw, nxt = n / w;
    const int threads = (tyv + 4) * 32;
    if (allow_dynamic_smem(fn, smem) != cudaSuccess) return false;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem) != cudaSuccess || occ < 1) return false;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return false;
    const int nyt = n / tyv;
    const long long tiles = (long long)nyt * nxt, units = tiles * n;
    long long blocks = 0;
    // whole groups of nxt blocks (the x tiles of a y tile, marching together)
    if (zr > 0) blocks = tiles * ((n + std::min(zr, n) - 1) / std::min(zr, n));
    else blocks = std::min((long long)sms * occ, units) / nxt * nxt;
    if (blocks < nxt) return false;
    const long long groups = blocks / nxt;
    cfg->ty = tyv;
    cfg->zr = (int)(((long long)nyt * n + groups - 1) / groups);
    cfg->nzc = (int)((groups + nyt - 1) / nyt);
    cfg->depth = d;
    cfg->threads = threads;
    cfg->maxt = threads;
    cfg->fast = 1;
    cfg->smem = smem;
    cfg->nyt = nyt;
    cfg->blocks = (int)blocks;
    cfg->nzl = 0;
    cfg->zbase = 0;
    cfg->s27 = 1;
    cfg->xt = 0;
    cfg->xw = 1;
    cfg->nxt = nxt;
    return true;
}

template <typename T>
cudaError_t launch_step27w(const Bufs<T>& b, const Model& M, DevScalars* sc, double* partials, const MarchConfig& cfg,
                           cudaStream_t st)
{
    size_t smem = 0;
    const void* fn = s27w_fn<T>(M.n, cfg.ty, cfg.depth, &smem);
    if (!fn) return cudaErrorInvalidValue;
    void* args[] = {(void*)&b, (void*)&M, (void*)&sc, (void*)&partials};
    return cudaLaunchKernel(fn, dim3(cfg.blocks), dim3(cfg.threads), args, cfg.smem, st);
}

template cudaError_t launch_step27w<float>(const Bufs<float>&, const Model&, DevScalars*, double*, const MarchConfig&,
                                           cudaStream_t);
template cudaError_t launch_step27w<double>(const Bufs<double>&, const Model&, DevScalars*, double*,
                                            const MarchConfig&, cudaStream_t);

} // namespace lat
