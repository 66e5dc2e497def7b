// lat_step27.cu -- the fused leapfrog step with the 27-point Laplacian of
// Sec. II.C (Patra and Karttunen: second-order accurate, fourth-order
// isotropic) on the shared-memory plane ring, FP32 and FP64.
//
// Same step and same ring as the 7-point plane-ring kernel (lat_march.cuh):
// a block owns full x rows, ty rows in y and a run of z planes; one thread owns
// one 16-byte vector of one row of the tile or of its halo (one row below, two
// above); planes arrive by per-thread asynchronous copies `depth` planes ahead.
//
// Laplacian. With the weights in units of 1/(30 dx^2) (faces 14, edges 12 x 3,
// corners 8 x 1) and, for each plane p of the 3x3x3 cube, the in-plane sums of
// exact differences from that plane's own centre C_p,
//   e_p = sum of the 4 face neighbours in the plane - 4 C_p,
//   k_p = sum of the 4 corner neighbours in the plane - 4 C_p,
// the stencil is
//   30 dx^2 L f = (14 e_z + 3 k_z) + (3 e_{z-1} + k_{z-1}) + (3 e_{z+1} + k_{z+1})
//                 + 30 ((C_{z-1} - c) + (C_{z+1} - c)),
// every term a sum of differences that are exact for f = const + small
// (Sterbenz), as in the 7-point kernel.
//
// Gradient average of the new fields (eq. scale): -<g L g> equals the mean over
// sites of the weighted squared differences over the 13 neighbour pairs each
// site owns. The owned offsets all have dy >= 0, so the one look-ahead row in
// +y that the ring already provides suffices: per site four pairs in its plane
// P, six to plane P + 1 and, for the site above it in P + 1, three back to P
// (rows y, y + 1 of planes P and P + 1). The new-field planes are kept in a
// triple buffer so that the pairs of plane P = k - 2 are summed at plane k
// without another barrier; the last pair of planes of a run is summed after it.
#include <algorithm>

#include "lat_kernels.h"
#include "lat_march.cuh"

namespace lat {

namespace {

template <typename T>
struct RowV {
    typename PK<T>::P v[PK<T>::NP];
    T l, r;   // the row's values left of the vector's first site and right of its last
};

// One row vector and its x neighbours: from the adjacent lanes where they hold
// the same row, else from shared memory (dl, dr: offsets of the periodic
// neighbours). Every lane of the warp calls this (shuffles).
template <typename T>
__device__ __forceinline__ void load_row(const T* p, RowV<T>& R, bool nbl, bool nbr, int dl, int dr)
{
    constexpr int NP = PK<T>::NP;
    PK<T>::ld(p, R.v);
    R.l = __shfl_up_sync(0xffffffffu, hi2(R.v[NP - 1]), 1);
    R.r = __shfl_down_sync(0xffffffffu, lo2(R.v[0]), 1);
    if (!nbl) R.l = p[dl];
    if (!nbr) R.r = p[dr];
}

// the row shifted by one site: o[i] holds the value at x_i - 1 (shl) or x_i + 1 (shr)
template <typename T>
__device__ __forceinline__ void shl(const RowV<T>& R, typename PK<T>::P (&o)[PK<T>::NP])
{
    if constexpr (PK<T>::NP == 2) {
        T c0, c1, c2, c3;
        un2(R.v[0], c0, c1);
        un2(R.v[1], c2, c3);
        o[0] = mk2(R.l, c0);
        o[1] = mk2(c1, c2);
    } else {
        o[0] = mk2(R.l, lo2(R.v[0]));
    }
}
template <typename T>
__device__ __forceinline__ void shr(const RowV<T>& R, typename PK<T>::P (&o)[PK<T>::NP])
{
    if constexpr (PK<T>::NP == 2) {
        T c0, c1, c2, c3;
        un2(R.v[0], c0, c1);
        un2(R.v[1], c2, c3);
        o[0] = mk2(c1, c2);
        o[1] = mk2(c3, R.r);
    } else {
        o[0] = mk2(hi2(R.v[0]), R.r);
    }
}

// e and k of one plane at this thread's sites: C the centre row, Ym and Yp the
// rows y - 1 and y + 1 of the same plane
template <typename T>
__device__ __forceinline__ void plane_ek(const RowV<T>& C, const RowV<T>& Ym, const RowV<T>& Yp,
                                         typename PK<T>::P (&e)[PK<T>::NP], typename PK<T>::P (&k)[PK<T>::NP])
{
    typedef typename PK<T>::P P;
    constexpr int NP = PK<T>::NP;
    P cl[NP], cr[NP], ml[NP], mr[NP], pl[NP], pr[NP];
    shl(C, cl);
    shr(C, cr);
    shl(Ym, ml);
    shr(Ym, mr);
    shl(Yp, pl);
    shr(Yp, pr);
#pragma unroll
    for (int v = 0; v < NP; v++) {
        const P c = C.v[v];
        e[v] = add2(add2(sub2(cl[v], c), sub2(cr[v], c)), add2(sub2(Ym.v[v], c), sub2(Yp.v[v], c)));
        k[v] = add2(add2(sub2(ml[v], c), sub2(mr[v], c)), add2(sub2(pl[v], c), sub2(pr[v], c)));
    }
}

// Per-thread sums of the new fields: the squared differences of each field
// over its owned pairs by weight class (14, 3, 1) and the potential sums of
// lat_site.cuh.
template <typename T>
struct Sums27 {
    typename PK<T>::P w14[2], w3[2], w1[2], vd, vi;
    __device__ void zero()
    {
        const typename PK<T>::P z = mk2(T(0), T(0));
        w14[0] = w14[1] = w3[0] = w3[1] = w1[0] = w1[1] = vd = vi = z;
    }
    __device__ void totals(bool quartic, double v[kSums]) const
    {
        for (int f = 0; f < 2; f++)
            v[f] = 14.0 * ((double)lo2(w14[f]) + (double)hi2(w14[f])) + 3.0 * ((double)lo2(w3[f]) + (double)hi2(w3[f]))
                   + ((double)lo2(w1[f]) + (double)hi2(w1[f]));
        v[2] = ((double)lo2(vd) + (double)hi2(vd)) * (double)site_vsum_factor<T>(quartic);
        v[3] = 0.5 * ((double)lo2(vi) + (double)hi2(vi));
    }
};

template <typename T>
__device__ __forceinline__ typename PK<T>::P sq_acc(typename PK<T>::P a, typename PK<T>::P b, typename PK<T>::P acc)
{
    const typename PK<T>::P d = sub2(a, b);
    return fma2(d, d, acc);
}

// Pairs of new-field plane P (Gp) with plane P + 1 (Gu) at this thread's own
// row: rows j, j + 1 (o1 = the row stride for the owned rows, 0 for the others
// so that they stay inside the plane). Rows j, j + 1 of plane P are those of the previous
// call's plane P + 1 when `carried` (kept in c0r, c1r); this call leaves its
// plane P + 1 rows there. Every lane calls this.
template <typename T>
__device__ __forceinline__ void pair_sums(const T* Gp, const T* Gu, uint32_t fieldG, int o1, bool own,
                                          const SiteCoefs<T>& K, bool nbl, bool nbr, int dl, int dr, bool carried,
                                          RowV<T> (&c0r)[2], RowV<T> (&c1r)[2], Sums27<T>& A)
{
    typedef typename PK<T>::P P;
    constexpr int NP = PK<T>::NP;
    P c0[NP];
#pragma unroll
    for (int f = 0; f < 2; f++) {
        const T* gu = Gu + f * fieldG;
        RowV<T> p0, p1, u0, u1;
        if (carried) {
            p0 = c0r[f];
            p1 = c1r[f];
        } else {
            const T* gp = Gp + f * fieldG;
            load_row(gp, p0, nbl, nbr, dl, dr);
            load_row(gp + o1, p1, nbl, nbr, dl, dr);
        }
        load_row(gu, u0, nbl, nbr, dl, dr);
        load_row(gu + o1, u1, nbl, nbr, dl, dr);
        c0r[f] = u0;
        c1r[f] = u1;
        if (own) {
            P p0r[NP], p1l[NP], p1r[NP], u0l[NP], u0r[NP], u1l[NP], u1r[NP];
            shr(p0, p0r);
            shl(p1, p1l);
            shr(p1, p1r);
            shl(u0, u0l);
            shr(u0, u0r);
            shl(u1, u1l);
            shr(u1, u1r);
            P a14 = A.w14[f], a3 = A.w3[f], a1 = A.w1[f];
#pragma unroll
            for (int v = 0; v < NP; v++) {
                const P c = p0.v[v], cu = u0.v[v];
                // site (x, y, P): in its plane (1,0,0) (0,1,0) (1,1,0) (-1,1,0); to P + 1
                // (0,0,1) (+-1,0,1) (0,1,1) (+-1,1,1); site (x, y, P + 1): (0,1,-1) (+-1,1,-1)
                a14 = sq_acc<T>(p0r[v], c, sq_acc<T>(p1.v[v], c, sq_acc<T>(u0.v[v], c, a14)));
                a3 = sq_acc<T>(p1r[v], c, sq_acc<T>(p1l[v], c, sq_acc<T>(u0r[v], c, sq_acc<T>(u0l[v], c,
                         sq_acc<T>(u1.v[v], c, sq_acc<T>(p1.v[v], cu, a3))))));
                a1 = sq_acc<T>(u1r[v], c, sq_acc<T>(u1l[v], c, sq_acc<T>(p1r[v], cu, sq_acc<T>(p1l[v], cu, a1))));
                if (f == 0) c0[v] = c;
            }
            A.w14[f] = a14;
            A.w3[f] = a3;
            A.w1[f] = a1;
            if (f == 1) {
#pragma unroll
                for (int v = 0; v < NP; v++) site_vsum<T>(K, c0[v], p0.v[v], A.vd, A.vi);
            }
        }
    }
}

// Plane aggregates at this thread's sites: centre C, q = 3 e + k (the plane's
// part when it is the plane below or above) and r = 14 e + 3 k (its part when it
// is the centre plane). F points at this thread's vector of the plane; ry is
// the row step (0 for threads that only stage). Every lane calls this.
template <typename T>
__device__ __forceinline__ void plane_aggr(const T* F, int ry, bool nbl, bool nbr, int dl, int dr,
                                           typename PK<T>::P (&C)[PK<T>::NP], typename PK<T>::P (&q)[PK<T>::NP],
                                           typename PK<T>::P (&r)[PK<T>::NP])
{
    typedef typename PK<T>::P P;
    constexpr int NP = PK<T>::NP;
    RowV<T> c, ym, yp;
    load_row(F, c, nbl, nbr, dl, dr);
    load_row(F - ry, ym, nbl, nbr, dl, dr);
    load_row(F + ry, yp, nbl, nbr, dl, dr);
    P e[NP], k[NP];
    plane_ek(c, ym, yp, e, k);
    const P c3 = mk2(T(3), T(3)), c14 = mk2(T(14), T(14));
#pragma unroll
    for (int v = 0; v < NP; v++) {
        C[v] = c.v[v];
        q[v] = fma2(c3, e[v], k[v]);
        r[v] = fma2(c14, e[v], mul2(c3, k[v]));
    }
}

// March planes [z0, z0 + nz) of tile (xt, yt) through the ring S (the ring of
// the 7-point kernel followed by three new-field planes). A tile is W columns
// (x0 = xt W) by ty rows. Each shared-memory row holds the tile's W columns with
// one 16-byte vector on either side (the columns just left of x0 and just right
// of x0 + W, periodic in x): the threads of those halo vectors stage them and
// also kick and drift them, so that the new fields one column beyond the tile
// are at hand for the pairs of the sums; only the tile's own sites are stored.
template <typename T>
__device__ void march_segment27(const MarchLattice<T>& L, int xt, int W, int yt, int z0, int nz, T* S, Sums27<T>& A,
                                bool first)
{
    typedef typename PK<T>::P P;
    constexpr int NP = PK<T>::NP;
    constexpr int VW = 2 * NP;
    const int n = L.n, ty = L.ty, D = L.depth;
    const int Qh = W / VW + 2;                             // vectors per staged row
    const int RW = W + 2 * VW;                             // elements per staged row
    const int t = threadIdx.x;
    const int rho_raw = t / Qh;
    const bool live = rho_raw < ty + 3;                    // threads past the tile only join the barriers
    const int rho = min(rho_raw, ty + 2);
    const int xi = live ? t - rho_raw * Qh : 0;            // vector within the staged row
    const int xs = xi * VW;
    const bool comp = live && rho >= 1 && rho <= ty + 1;   // owned rows and the look-ahead row, halo vectors included
    const bool ownrow = comp && rho <= ty;
    const bool own = ownrow && xi >= 1 && xi <= Qh - 2;
    // x neighbours: adjacent vectors of the staged row (contiguous); the outer
    // neighbours of the halo vectors are not staged and not needed (read in place)
    const int dl = xi > 0 ? -1 : 0;
    const int dr = xi < Qh - 1 ? VW : 0;
    const RingGeom R = ring_geom(RW, ty, D);
    const uint32_t offF = (uint32_t)rho * RW + xs;
    const uint32_t offP = (uint32_t)(comp ? rho - 1 : 0) * RW + xs;
    const int ry = comp ? RW : 0;      // row step to y +- 1 (0 for threads that only stage)
    // row step to j + 1 in the sums: the same for every vector of a row (the halo
    // vectors of an owned row feed their neighbours' shuffles)
    const int o1 = ownrow ? RW : 0;
    const uint32_t nn = (uint32_t)n * n;
    const int gx = wrapn(xt * W - VW + xs, n);
    const uint32_t rowg = (uint32_t)wrapn(yt * ty - 1 + rho, n) * n + gx;

    auto fetch_f = [&](int zrel, int slot) {
        const uint32_t gi = L.plane(z0 + zrel) * nn + rowg;
        T* d = S + (uint32_t)slot * R.slotF + offF;
        cp_async16(d, L.f0 + gi);
        cp_async16(d + R.fieldF, L.f1 + gi);
    };
    auto fetch_p = [&](int zrel, int slot) {
        const uint32_t gi = L.plane(z0 + zrel) * nn + rowg;
        T* d = S + R.p0 + (uint32_t)slot * R.slotP + offP;
        cp_async16(d, L.p0 + gi);
        cp_async16(d + R.fieldP, L.p1 + gi);
    };
    const int lane = t & 31;
    const bool nbl = xi > 0 && lane > 0, nbr = xi < Qh - 1 && lane < 31;
    auto addm = [](int a, int b, int m) { return a + b >= m ? a + b - m : a + b; };
    T* const G0 = S + R.g0;            // three new-field planes of R.planeG elements

    if (!first) __syncthreads();
    if (live) {
        fetch_f(-1, 0);
        fetch_f(0, 1);
        fetch_f(1, 2);
        if (comp) fetch_p(0, 0);
    }
    cp_async_commit();
    for (int j = 1; j < D; j++) {
        if (live && 1 + j <= nz + 1) fetch_f(1 + j, 2 + j);
        if (comp && j <= nz) fetch_p(j, j);
        cp_async_commit();
    }
    int sf = 0, sp = 0, sg = 0;        // k mod (D+3), k mod (D+1), k mod 3

    const P dtcl2 = mk2(L.K.dtcl, L.K.dtcl), dtcf2 = mk2(L.K.dtcf, L.K.dtcf);
    const P c30 = mk2(T(30), T(30));
    P Cm[2][NP], qm[2][NP], Cc[2][NP], qc[2][NP], rc[2][NP];   // aggregates of planes z - 1 and z
    RowV<T> gr0[2], gr1[2];   // rows j, j + 1 of the newest new-field plane summed so far
    for (int k = 0; k <= nz; k++) {
        const bool ahead = k == nz;
        const int z = z0 + k;
        cp_async_wait(D - 1);
        __syncthreads();
        if (live && k + 1 + D <= nz + 1) fetch_f(k + 1 + D, addm(sf, D + 2, R.rf));
        if (comp && k + D <= nz) fetch_p(k + D, addm(sp, D, R.rp));
        cp_async_commit();

        const T* Fm = S + (uint32_t)sf * R.slotF + offF;
        const T* Fc = S + (uint32_t)addm(sf, 1, R.rf) * R.slotF + offF;
        const T* Fp = S + (uint32_t)addm(sf, 2, R.rf) * R.slotF + offF;
        const T* Pc = S + R.p0 + (uint32_t)sp * R.slotP + offP;
        sf = addm(sf, 1, R.rf);
        sp = addm(sp, 1, R.rp);
        T* Gw = G0 + (uint32_t)sg * R.planeG;
        const T* Gm1 = G0 + (uint32_t)addm(sg, 2, 3) * R.planeG;   // plane k - 1
        const T* Gm2 = G0 + (uint32_t)addm(sg, 1, 3) * R.planeG;   // plane k - 2
        sg = addm(sg, 1, 3);

        // kick and drift of rows 1 .. ty + 1 (owned and look-ahead) of plane z:
        // the aggregates of planes z - 1 and z come from the two previous planes
        // (computed here for the first plane of the run), those of z + 1 are new
        P pn[2][NP];
        if (k == 0) {
#pragma unroll
            for (int f = 0; f < 2; f++) {
                P rdummy[NP];
                plane_aggr<T>(Fm + f * R.fieldF, ry, nbl, nbr, dl, dr, Cm[f], qm[f], rdummy);
                plane_aggr<T>(Fc + f * R.fieldF, ry, nbl, nbr, dl, dr, Cc[f], qc[f], rc[f]);
            }
        }
#pragma unroll
        for (int f = 0; f < 2; f++) {
            P Cp[NP], qp[NP], rp[NP], pv[NP];
            plane_aggr<T>(Fp + f * R.fieldF, ry, nbl, nbr, dl, dr, Cp, qp, rp);
            PK<T>::ld(Pc + f * R.fieldP, pv);
#pragma unroll
            for (int v = 0; v < NP; v++) {
                const P c = Cc[f][v];
                const P lap = fma2(c30, add2(sub2(Cm[f][v], c), sub2(Cp[v], c)), add2(rc[f][v], add2(qm[f][v], qp[v])));
                pn[f][v] = fma2(dtcl2, lap, fma2(dtcf2, c, pv[v]));
                Cm[f][v] = c;
                qm[f][v] = qc[f][v];
                Cc[f][v] = Cp[v];
                qc[f][v] = qp[v];
                rc[f][v] = rp[v];
            }
        }
        if (comp) {
            P g[2][NP];
            // potential part of the kick and the drift of plane z (shifted down
            // above) (lat_site.cuh)
#pragma unroll
            for (int v = 0; v < NP; v++) site_kick_drift<T>(L.K, Cm[0][v], Cm[1][v], pn[0][v], pn[1][v], g[0][v], g[1][v]);
            if (own && !ahead) {
                const uint32_t gi = L.plane(z) * nn + rowg;
                PK<T>::st(L.op0 + gi, pn[0]);
                PK<T>::st(L.op1 + gi, pn[1]);
                PK<T>::st(L.of0 + gi, g[0]);
                PK<T>::st(L.of1 + gi, g[1]);
            }
            PK<T>::st(Gw + offP, g[0]);
            PK<T>::st(Gw + R.fieldG + offP, g[1]);
        }

        // pairs of planes k - 2 and k - 1 (both written before the barrier above)
        if (k >= 2)
            pair_sums(Gm2 + offP, Gm1 + offP, R.fieldG, o1, own, L.K, nbl, nbr, dl, dr, false, gr0, gr1, A);
    }
    // the last pair: planes nz - 1 and nz (the look-ahead plane)
    __syncthreads();
    {
        const T* Gl = G0 + (uint32_t)addm(sg, 2, 3) * R.planeG;   // plane nz (sg = (nz + 1) mod 3)
        const T* Gb = G0 + (uint32_t)addm(sg, 1, 3) * R.planeG;   // plane nz - 1
        pair_sums(Gb + offP, Gl + offP, R.fieldG, o1, own, L.K, nbl, nbr, dl, dr, false, gr0, gr1, A);
    }
}

struct Args27 {
    int ty, nyt, depth;
    int nxt, W;     // x tiles per row and their width
};

template <typename T, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) step27_kernel(Bufs<T> B, Model M, DevScalars* sc, double* partials, Args27 G)
{
    __shared__ double red[32 * kSums];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (sc->status != LAT_OK) return;
    T* const S = reinterpret_cast<T*>(smem_raw);
    const int n = M.n;
    const bool par = (sc->step & 1) != 0;
    MarchLattice<T> L;
    L.f0 = par ? B.f[1][0] : B.f[0][0];
    L.f1 = par ? B.f[1][1] : B.f[0][1];
    L.p0 = par ? B.p[1][0] : B.p[0][0];
    L.p1 = par ? B.p[1][1] : B.p[0][1];
    L.of0 = par ? B.f[0][0] : B.f[1][0];
    L.of1 = par ? B.f[0][1] : B.f[1][1];
    L.op0 = par ? B.p[0][0] : B.p[1][0];
    L.op1 = par ? B.p[0][1] : B.p[1][1];
    L.n = n;
    L.ty = G.ty;
    L.depth = G.depth;
    L.K = site_coefs<T>(sc, M.beta);
    L.periodic = true;
    L.zbase = 0;
    Sums27<T> A;
    A.zero();

    // The nxt x tiles of a y tile go to nxt consecutive blocks (a group) that
    // take the same (y tile, z plane) units: the groups share the nyt * n units
    // equally, and the blocks of a group march the same planes at the same
    // time, so the 16-byte halo vectors each tile reads from its x neighbours lie
    // in memory lines the neighbouring block is reading too, and come from L2
    // instead of a second DRAM read of the whole line.
    const int ngroups = gridDim.x / G.nxt;
    const int grp = blockIdx.x / G.nxt, xt = blockIdx.x - grp * G.nxt;
    const long long U = (long long)G.nyt * n;
    long long u = (long long)grp * U / ngroups;
    const long long uend = ((long long)grp + 1) * U / ngroups;
    for (bool first = true; u < uend; first = false) {
        const int yt = (int)(u / n);
        const int z0 = (int)(u - (long long)yt * n);
        const int nz = (int)min((long long)(n - z0), uend - u);
        u += nz;
        march_segment27(L, xt, G.W, yt, z0, nz, S, A, first);
    }
    double v[kSums];
    A.totals(L.K.quartic, v);
    finish_block(M, sc, partials, v, red, true);
}

constexpr int kMaxts27[] = {256, 512, 768, 1024};

int maxt27_for(int threads)
{
    for (int m : kMaxts27)
        if (threads <= m) return m;
    return 0;
}

template <typename T>
const void* step27_fn(int maxt)
{
    switch (maxt) {
    case 256: return (const void*)step27_kernel<T, 256>;
    case 512: return (const void*)step27_kernel<T, 512>;
    case 768: return (const void*)step27_kernel<T, 768>;
    default: return (const void*)step27_kernel<T, 1024>;
    }
}

size_t smem27(int rw, int esize, int ty, int depth)
{
    // the ring of the 7-point kernel over rows of rw elements, with three
    // new-field planes instead of two
    return (size_t)esize * rw * ((depth + 3) * 2 * (ty + 3) + (depth + 1) * 2 * (ty + 1) + 3 * 2 * (ty + 1));
}

// x tiles per row: the fewest that keep a tile at most 16 vectors wide, among
// those that divide the row into whole vectors (narrow tiles leave room in 512
// threads for taller ones: 16 rows of 16 vectors recompute fewer halo and
// look-ahead sites per owned site than 4 rows of 64, and measured 11 % faster)
int nxt_for(int n, int vw)
{
    const int q = n / vw;
    for (int nxt = (q + 15) / 16; nxt <= q; nxt++)
        if (q % nxt == 0) return nxt;
    return q;
}

bool geom27(int n, int esize, int ty, int zr, int depth, MarchConfig* cfg)
{
    const int vw = 16 / esize;
    if (n % 4 != 0 || n < 4 || ty < 1 || ty > n || n % ty != 0) return false;
    if (depth < 1 || depth > 4) return false;
    const int nxt = nxt_for(n, vw);
    const int W = n / nxt;
    int threads = (ty + 3) * (W / vw + 2);
    threads = ((threads + 31) / 32) * 32;
    if (threads > 1024) return false;
    const size_t smem = smem27(W + 2 * vw, esize, ty, depth);
    if (smem > 227 * 1024 - 2048) return false;
    const int maxt = maxt27_for(threads);
    const void* fn = esize == 4 ? step27_fn<float>(maxt) : step27_fn<double>(maxt);
    if (allow_dynamic_smem(fn, smem) != cudaSuccess) return false;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem) != cudaSuccess || occ < 1) return false;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return false;
    const int nyt = n / ty;
    const long long tiles = (long long)nyt * nxt;
    const long long units = tiles * n;
    long long blocks = 0;
    // whole groups of nxt blocks (the x tiles of a y tile, marching together)
    if (zr > 0) blocks = tiles * ((n + std::min(zr, n) - 1) / std::min(zr, n));
    else blocks = std::min((long long)sms * occ, units) / nxt * nxt;
    const long long groups = blocks / nxt;
    cfg->ty = ty;
    cfg->zr = (int)(((long long)nyt * n + groups - 1) / groups);
    cfg->nzc = (int)((groups + nyt - 1) / nyt);
    cfg->depth = depth;
    cfg->threads = threads;
    cfg->maxt = maxt;
    cfg->fast = 0;
    cfg->smem = smem;
    cfg->nyt = nyt;
    cfg->blocks = (int)blocks;
    cfg->nzl = 0;
    cfg->zbase = 0;
    cfg->s27 = 1;
    cfg->nxt = nxt;
    return true;
}

} // namespace

bool march27_config(int n, int elem_bytes, int ty, int zr, int depth, MarchConfig* cfg)
{
    const int d = depth > 0 ? depth : 1;
    if (ty > 0) return geom27(n, elem_bytes, ty, zr, d, cfg);
    // default: the tallest tile whose block stays within 512 threads (registers
    // for the 27-point arithmetic), else the tallest that fits at all
    const int tys[] = {16, 8, 4, 2, 1};
    const int vw = 16 / elem_bytes;
    const int qh = n / nxt_for(n, vw) / vw + 2;
    for (int t : tys)
        if ((t + 3) * qh <= 512 && geom27(n, elem_bytes, t, zr, d, cfg)) return true;
    for (int t : tys)
        if (geom27(n, elem_bytes, t, zr, d, cfg)) return true;
    return false;
}

template <typename T>
cudaError_t launch_step27(const Bufs<T>& b, const Model& M, DevScalars* sc, double* partials, const MarchConfig& cfg,
                          cudaStream_t st)
{
    Args27 G{cfg.ty, cfg.nyt, cfg.depth, cfg.nxt, M.n / cfg.nxt};
    switch (cfg.maxt) {
    case 256: step27_kernel<T, 256><<<cfg.blocks, cfg.threads, cfg.smem, st>>>(b, M, sc, partials, G); break;
    case 512: step27_kernel<T, 512><<<cfg.blocks, cfg.threads, cfg.smem, st>>>(b, M, sc, partials, G); break;
    case 768: step27_kernel<T, 768><<<cfg.blocks, cfg.threads, cfg.smem, st>>>(b, M, sc, partials, G); break;
    default: step27_kernel<T, 1024><<<cfg.blocks, cfg.threads, cfg.smem, st>>>(b, M, sc, partials, G); break;
    }
    return cudaGetLastError();
}

template cudaError_t launch_step27<float>(const Bufs<float>&, const Model&, DevScalars*, double*, const MarchConfig&,
                                          cudaStream_t);
template cudaError_t launch_step27<double>(const Bufs<double>&, const Model&, DevScalars*, double*,
                                           const MarchConfig&, cudaStream_t);

} // namespace lat
