// lat_march.cuh -- one z-march segment of the fused leapfrog step on a shared-
// memory plane ring (Sec. II.B, eq. evo with eq. scalar-evo, and the sums of the
// new fields for eq. scale). Used by the single-lattice plane-ring kernel
// (lat_step_march.cu) and by the persistent ensemble kernel (lat_batch.cu).
//
// A block owns full x rows, `ty` rows in y and a run of planes in z. One thread
// owns one 16-byte vector (4 floats or 2 doubles) of one row of the tile or of
// its halo (one row below, two above: the second for the look-ahead rim). Planes
// are staged in the ring by per-thread 16-byte asynchronous copies (cp.async)
// issued `depth` planes ahead; one barrier per plane. FP32 arithmetic is done
// on packed f32x2 pairs. The forward differences of the new fields in x and y,
// and their potential, are summed one plane later from a double-buffered shared
// copy of the new fields; the z difference uses the previous plane's new fields.
#pragma once

#include "lat_async.cuh"
#include "lat_common.cuh"
#include "lat_pairs.cuh"
#include "lat_site.cuh"

namespace lat {

// Shared ring for prefetch depth D: D+3 field-plane slots [slot][field][ty+3
// rows][n] (planes z-1, z, z+1 in use, D planes in flight), D+1 momentum slots
// [slot][field][ty+1 rows][n], 2 new-field planes [buf][field][ty+1 rows][n].
// Offsets in elements.
struct RingGeom {
    uint32_t fieldF, slotF, fieldP, slotP, fieldG, planeG, p0, g0;
    int rf, rp;
};

__host__ __device__ inline RingGeom ring_geom(int n, int ty, int depth)
{
    RingGeom R;
    R.rf = depth + 3;
    R.rp = depth + 1;
    R.fieldF = (uint32_t)(ty + 3) * n;
    R.slotF = 2 * R.fieldF;
    R.fieldP = (uint32_t)(ty + 1) * n;
    R.slotP = 2 * R.fieldP;
    R.fieldG = R.fieldP;
    R.planeG = R.slotP;
    R.p0 = R.rf * R.slotF;
    R.g0 = R.p0 + R.rp * R.slotP;
    return R;
}

// Elements of the ring.
__host__ __device__ inline size_t ring_elems(int n, int ty, int depth)
{
    const RingGeom R = ring_geom(n, ty, depth);
    return (size_t)R.g0 + 2 * (size_t)R.planeG;
}

// One lattice during one step, as a march segment sees it.
template <typename T>
struct MarchLattice {
    const T *f0, *f1, *p0, *p1;   // fields at the field time and momenta (read)
    T *of0, *of1, *op0, *op1;     // the other ping-pong set (written)
    int n, ty, depth;
    SiteCoefs<T> K;                      // the step's coefficients (lat_site.cuh)
    // z storage: periodic (plane z stored at z mod n) or a z-slab whose arrays
    // hold plane z at z + zbase (halo planes below and above the owned ones)
    bool periodic;
    int zbase;
    __device__ __forceinline__ uint32_t plane(int z) const
    {
        return (uint32_t)(periodic ? wrapn(z, n) : z + zbase);
    }
};

// Per-thread sums of the new fields (packed pairs): forward-difference
// gradients of each field and the potential sums of lat_site.cuh (factors
// applied at the end).
template <typename T>
struct MarchSums {
    typename PK<T>::P accg0, accg1, accvd, accvi;
    __device__ void zero()
    {
        accg0 = mk2(T(0), T(0));
        accg1 = accg0;
        accvd = accg0;
        accvi = accg0;
    }
    // the four sums of this thread in the element type (1/beta and 1/2 are powers
    // of two, exact); the potential sums are taken about the homogeneous mode
    __device__ void totals(bool quartic, T v[kSums]) const
    {
        v[0] = lo2(accg0) + hi2(accg0);
        v[1] = lo2(accg1) + hi2(accg1);
        v[2] = (lo2(accvd) + hi2(accvd)) * site_vsum_factor<T>(quartic);
        v[3] = T(0.5) * (lo2(accvi) + hi2(accvi));
    }
};

// March planes [z0, z0 + nz) of y tile yt (rows yt*ty .. yt*ty+ty-1) through the
// ring S: kick and drift of the owned sites, written to the other set, and the
// sums of the new fields of those sites added to A. `first`: no earlier segment
// of this block is still reading the ring. SPLIT: the lattice may store phi
// split (lat_site.cuh); false compiles the forms for phi stored whole.
template <typename T, bool SPLIT = true>
__device__ void march_segment(const MarchLattice<T>& L, int yt, int z0, int nz, T* S, MarchSums<T>& A, bool first)
{
    typedef typename PK<T>::P P;
    constexpr int NP = PK<T>::NP;
    constexpr int VW = 2 * NP;
    const int n = L.n, ty = L.ty, D = L.depth, Q = n / VW;
    const int t = threadIdx.x;
    const int rho_raw = t / Q;
    const bool live = rho_raw < ty + 3;                    // threads past the tile only join the barriers
    const int rho = min(rho_raw, ty + 2);
    const int x = live ? (t - rho_raw * Q) * VW : 0;
    const bool comp = live && rho >= 1 && rho <= ty + 1;   // computes a new vector (owned rows + look-ahead row)
    const bool own = live && rho >= 1 && rho <= ty;
    const int dl = x == 0 ? n - 1 : -1;                     // left neighbour of the first site (periodic)
    const int dr = x + VW == n ? VW - n : VW;                // right neighbour of the last site
    const RingGeom R = ring_geom(n, ty, D);
    const uint32_t offF = (uint32_t)rho * n + x;            // this vector in a field plane
    const uint32_t offP = (uint32_t)(comp ? rho - 1 : 0) * n + x;   // in a momentum / new-field plane
    const uint32_t nn = (uint32_t)n * n;
    const uint32_t rowg = (uint32_t)wrapn(yt * ty - 1 + rho, n) * n + x;

    // copies of this thread's vectors of plane z0 + zrel: f into field slot
    // (zrel + 1) mod (D+3), momenta into momentum slot zrel mod (D+1); the slot
    // is passed in (kept as running counters, no division in the loop)
    auto fetch_f = [&](int zrel, int slot) {          // zrel in [-1, nz + 1]
        const uint32_t gi = L.plane(z0 + zrel) * nn + rowg;
        T* d = S + (uint32_t)slot * R.slotF + offF;
        cp_async16(d, L.f0 + gi);
        cp_async16(d + R.fieldF, L.f1 + gi);
    };
    auto fetch_p = [&](int zrel, int slot) {          // zrel in [0, nz]
        const uint32_t gi = L.plane(z0 + zrel) * nn + rowg;
        T* d = S + R.p0 + (uint32_t)slot * R.slotP + offP;
        cp_async16(d, L.p0 + gi);
        cp_async16(d + R.fieldP, L.p1 + gi);
    };
    // x neighbours in the adjacent lanes (same row, not wrapped), else shared memory
    const int lane = t & 31;
    const int qv = x / VW;
    const bool nbl = qv > 0 && lane > 0, nbr = qv < Q - 1 && lane < 31;
    auto addm = [](int a, int b, int m) { return a + b >= m ? a + b - m : a + b; };

    // the previous segment's last plane is read by every thread before the
    // prologue below refills the ring
    if (!first) __syncthreads();
    // prologue: group 0 = planes z0-1, z0, z0+1 and momenta of z0; group j < D =
    // plane z0+1+j and momenta of z0+j. Iteration k then commits group D+k
    // (plane z0+1+D+k, momenta z0+D+k) and waits for group k first.
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
    int sf = 0, sp = 0;          // k mod (D+3), k mod (D+1)

    for (int k = 0; k <= nz; k++) {
        const bool ahead = k == nz;
        const int z = z0 + k;                 // == n only on the look-ahead plane of the last chunk
        cp_async_wait(D - 1);
        __syncthreads();
        // prefetch into the slots released by plane k-1 (every thread has passed
        // the barrier above)
        if (live && k + 1 + D <= nz + 1) fetch_f(k + 1 + D, addm(sf, D + 2, R.rf));
        if (comp && k + D <= nz) fetch_p(k + D, addm(sp, D, R.rp));
        cp_async_commit();

        const T* Fm = S + (uint32_t)sf * R.slotF;
        const T* Fc = S + (uint32_t)addm(sf, 1, R.rf) * R.slotF;
        const T* Fp = S + (uint32_t)addm(sf, 2, R.rf) * R.slotF;
        const T* Pc = S + R.p0 + (uint32_t)sp * R.slotP;
        sf = addm(sf, 1, R.rf);
        sp = addm(sp, 1, R.rp);
        T* Gw = S + R.g0 + (k & 1) * R.planeG;
        const T* Gr = S + R.g0 + ((k + 1) & 1) * R.planeG;

        // centre vectors and their x neighbours (every lane takes part in the
        // shuffles; halo rows load harmlessly)
        P cen[2][NP];
        T lefts[2], rights[2];
#pragma unroll
        for (int f = 0; f < 2; f++) {
            const T* Ff = Fc + f * R.fieldF + offF;
            PK<T>::ld(Ff, cen[f]);
            lefts[f] = __shfl_up_sync(0xffffffffu, hi2(cen[f][NP - 1]), 1);
            rights[f] = __shfl_down_sync(0xffffffffu, lo2(cen[f][0]), 1);
            if (!nbl) lefts[f] = Ff[dl];
            if (!nbr) rights[f] = Ff[dr];
        }
        P g[2][NP];
        if (comp && !(ahead && rho == ty + 1)) {
            P pn[2][NP];
#pragma unroll
            for (int f = 0; f < 2; f++) {
                const T* Ff = Fc + f * R.fieldF + offF;
                P up[NP], dn[NP], zm[NP], zp[NP], pv[NP], lft[NP], rgt[NP];
                PK<T>::ld(Ff - n, up);
                PK<T>::ld(Ff + n, dn);
                PK<T>::ld(Fm + f * R.fieldF + offF, zm);
                PK<T>::ld(Fp + f * R.fieldF + offF, zp);
                PK<T>::ld(Pc + f * R.fieldP + offP, pv);
                const T left = lefts[f], right = rights[f];
                if constexpr (NP == 2) {
                    T c0, c1, c2, c3;
                    un2(cen[f][0], c0, c1);
                    un2(cen[f][1], c2, c3);
                    lft[0] = mk2(left, c0);
                    lft[1] = mk2(c1, c2);
                    rgt[0] = lft[1];
                    rgt[1] = mk2(c3, right);
                } else {
                    lft[0] = mk2(left, lo2(cen[f][0]));
                    rgt[0] = mk2(hi2(cen[f][0]), right);
                }
                const P dtcl2 = mk2(L.K.dtcl, L.K.dtcl), dtcf2 = mk2(L.K.dtcf, L.K.dtcf);
#pragma unroll
                for (int v = 0; v < NP; v++) {
                    const P c = cen[f][v];
                    // Laplacian as a sum of neighbour differences: exact differences
                    // for f = const + small (Sterbenz)
                    const P lapu = add2(add2(add2(sub2(lft[v], c), sub2(rgt[v], c)),
                                             add2(sub2(up[v], c), sub2(dn[v], c))),
                                        add2(sub2(zm[v], c), sub2(zp[v], c)));
                    pn[f][v] = fma2(dtcl2, lapu, fma2(dtcf2, c, pv[v]));
                }
            }
            // potential part of the kick and the drift (lat_site.cuh)
#pragma unroll
            for (int v = 0; v < NP; v++) {
                if constexpr (SPLIT) site_kick_drift<T>(L.K, cen[0][v], cen[1][v], pn[0][v], pn[1][v], g[0][v], g[1][v]);
                else site_kick_drift_whole<T>(L.K, cen[0][v], cen[1][v], pn[0][v], pn[1][v], g[0][v], g[1][v]);
            }
            if (!ahead) {
                if (own) {
                    const uint32_t gi = L.plane(z) * nn + rowg;
                    PK<T>::st(L.op0 + gi, pn[0]);
                    PK<T>::st(L.op1 + gi, pn[1]);
                    PK<T>::st(L.of0 + gi, g[0]);
                    PK<T>::st(L.of1 + gi, g[1]);
                }
                PK<T>::st(Gw + offP, g[0]);
                PK<T>::st(Gw + R.fieldG + offP, g[1]);
            }
        }

        // sums over the owned rows of plane k-1 (x and y pairs, potential) and the
        // z pair (k-1, k), from the new fields written one plane ago
        if (k > 0) {
            P gq[2][NP];
            T xnexts[2];
#pragma unroll
            for (int f = 0; f < 2; f++) {
                const T* Gf = Gr + f * R.fieldG + offP;
                PK<T>::ld(Gf, gq[f]);
                xnexts[f] = __shfl_down_sync(0xffffffffu, lo2(gq[f][0]), 1);
                if (!nbr) xnexts[f] = Gf[dr];
            }
            if (own) {
#pragma unroll
            for (int f = 0; f < 2; f++) {
                const T* Gf = Gr + f * R.fieldG + offP;
                P yn[NP], xn[NP];
                PK<T>::ld(Gf + n, yn);
                const T xnext = xnexts[f];
                if constexpr (NP == 2) {
                    T a, b, c, d;
                    un2(gq[f][0], a, b);
                    un2(gq[f][1], c, d);
                    xn[0] = mk2(b, c);
                    xn[1] = mk2(d, xnext);
                } else {
                    xn[0] = mk2(hi2(gq[f][0]), xnext);
                }
                P acc = f == 0 ? A.accg0 : A.accg1;
#pragma unroll
                for (int v = 0; v < NP; v++) {
                    const P dxv = sub2(xn[v], gq[f][v]), dyv = sub2(yn[v], gq[f][v]), dzv = sub2(g[f][v], gq[f][v]);
                    acc = fma2(dxv, dxv, fma2(dyv, dyv, fma2(dzv, dzv, acc)));
                }
                if (f == 0) A.accg0 = acc;
                else A.accg1 = acc;
            }
#pragma unroll
            for (int v = 0; v < NP; v++) {
                if constexpr (SPLIT) site_vsum<T>(L.K, gq[0][v], gq[1][v], A.accvd, A.accvi);
                else site_vsum_whole<T>(L.K, gq[0][v], gq[1][v], A.accvd, A.accvi);
            }
            }
        }
    }
}

} // namespace lat
