// lat_site.cuh -- the per-site arithmetic of one leapfrog step that every step
// kernel shares: the potential part of the kick (Sec. II.B, eq. scalar-evo with
// V_pr = cdom f0^beta/beta + kappa f0^2 f1^2/2), the drift (eq. evo) and the
// potential sums of the new fields for eq. scale, on packed two-site pairs.
//
// Field 0 is stored as its fluctuation d about the homogeneous mode P of the
// scalar block (P = 0 when phi is stored whole, see DevScalars), field 1 whole.
// With u = P + d the potential force on the stored arrays is
//   phi: cdom (u^(beta-1) - P^(beta-1)) + kappa u chi^2,  chi: kappa u^2 chi,
// where u^3 - P^3 = d (u (u + P) + P^2); and the potential sums are taken as
//   sum (u^beta - P^beta) = sum d (u + P) (u^2 + P^2)   (beta = 4)
//                         = sum d (u + P)                (beta = 2),
//   sum u^2 chi^2,
// P^beta/beta being added once in FP64 (advance_scalars). None of these forms
// takes a difference of nearby numbers, so FP32 arithmetic on d keeps the
// relative precision of d. With P = 0 they are the plain f0^3, f0 f1^2, f0^2 f1
// and f0^beta of phi stored whole, rounded the same way.
#pragma once

#include "lat_common.cuh"
#include "lat_pairs.cuh"

namespace lat {

// The step's coefficients in the element type.
template <typename T>
struct SiteCoefs {
    T dtcl, dtcf, mdtcdom, mdtkap, dt;   // dt cL/dx^2, dt cF, -dt cdom, -dt kappa, dt
    T bg, bg2;                           // P and P^2 at the field time of the step
    T bgn, bgn2;                         // P' and P'^2 at the new field time
    bool quartic;                        // beta == 4
};

template <typename T>
__device__ __forceinline__ SiteCoefs<T> site_coefs(const DevScalars* sc, int beta)
{
    SiteCoefs<T> C;
    C.dtcl = step_coef<T>(sc, kDtCl);
    C.dtcf = step_coef<T>(sc, kDtCf);
    C.mdtcdom = step_coef<T>(sc, kMDtCdom);
    C.mdtkap = step_coef<T>(sc, kMDtKap);
    C.dt = step_coef<T>(sc, kDt);
    C.bg = step_coef<T>(sc, kBg);
    C.bg2 = step_coef<T>(sc, kBg2);
    C.bgn = step_coef<T>(sc, kBgNew);
    C.bgn2 = step_coef<T>(sc, kBgNew2);
    C.quartic = beta == 4;
    return C;
}

// Potential part of the kick and the drift for one pair of sites: pn0, pn1 hold
// f' + dt (cL Lap f + cF f) on entry and the new momenta on return; g0, g1 get
// the new fields. a0 = d (field 0 as stored), a1 = chi.
template <typename T>
__device__ __forceinline__ void site_kick_drift(const SiteCoefs<T>& C, typename PK<T>::P a0, typename PK<T>::P a1,
                                                typename PK<T>::P& pn0, typename PK<T>::P& pn1,
                                                typename PK<T>::P& g0, typename PK<T>::P& g1)
{
    typedef typename PK<T>::P P;
    const P bg = mk2(C.bg, C.bg), mdtkap = mk2(C.mdtkap, C.mdtkap), mdtcdom = mk2(C.mdtcdom, C.mdtcdom);
    const P u = add2(bg, a0);
    const P ue = mul2(u, a1);
    const P dom = C.quartic ? mul2(a0, fma2(u, add2(u, bg), mk2(C.bg2, C.bg2))) : a0;
    pn0 = fma2(mdtcdom, dom, fma2(mdtkap, mul2(ue, a1), pn0));
    pn1 = fma2(mdtkap, mul2(ue, u), pn1);
    const P dt = mk2(C.dt, C.dt);
    g0 = fma2(dt, pn0, a0);
    g1 = fma2(dt, pn1, a1);
}

// Scalar arithmetic without contraction, so that one site computed alone rounds
// exactly as the same site in a packed pair (add.rn, mul.rn and fma.rn of the
// f32x2 instructions act per element).
__device__ __forceinline__ float s_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float s_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float s_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float s_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double s_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double s_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double s_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double s_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

// site_kick_drift for one site, rounded as each element of the packed form.
template <typename T>
__device__ __forceinline__ void site_kick_drift1(const SiteCoefs<T>& C, T a0, T a1, T& pn0, T& pn1, T& g0, T& g1)
{
    const T u = s_add(C.bg, a0);
    const T ue = s_mul(u, a1);
    const T dom = C.quartic ? s_mul(a0, s_fma(u, s_add(u, C.bg), C.bg2)) : a0;
    pn0 = s_fma(C.mdtcdom, dom, s_fma(C.mdtkap, s_mul(ue, a1), pn0));
    pn1 = s_fma(C.mdtkap, s_mul(ue, u), pn1);
    g0 = s_fma(C.dt, pn0, a0);
    g1 = s_fma(C.dt, pn1, a1);
}

// Potential sums of one pair of new sites (d = field 0 as stored, e = chi) about
// the new homogeneous mode P', u = P' + d: accd += u^beta - P'^beta (times 1/beta
// later, site_vsum_factor), acci += u^2 e^2.
template <typename T>
__device__ __forceinline__ void site_vsum(const SiteCoefs<T>& C, typename PK<T>::P d, typename PK<T>::P e,
                                          typename PK<T>::P& accd, typename PK<T>::P& acci)
{
    typedef typename PK<T>::P P;
    const P bgn = mk2(C.bgn, C.bgn);
    const P u = add2(d, bgn);
    const P s = add2(u, bgn);
    if (C.quartic) accd = fma2(mul2(d, s), fma2(u, u, mk2(C.bgn2, C.bgn2)), accd);
    else accd = fma2(d, s, accd);
    const P ue = mul2(u, e);
    acci = fma2(ue, ue, acci);
}

// The same two helpers for a lattice that stores phi whole (P = P' = 0): the
// arithmetic of the general forms with P = 0, instruction for instruction, but
// without the mode's coefficients held in registers (kernels that are compiled
// for both use these when no lattice they step stores phi split).
template <typename T>
__device__ __forceinline__ void site_kick_drift_whole(const SiteCoefs<T>& C, typename PK<T>::P a0, typename PK<T>::P a1,
                                                      typename PK<T>::P& pn0, typename PK<T>::P& pn1,
                                                      typename PK<T>::P& g0, typename PK<T>::P& g1)
{
    typedef typename PK<T>::P P;
    const P mdtkap = mk2(C.mdtkap, C.mdtkap), mdtcdom = mk2(C.mdtcdom, C.mdtcdom);
    const P ue = mul2(a0, a1);
    const P dom = C.quartic ? mul2(a0, mul2(a0, a0)) : a0;
    pn0 = fma2(mdtcdom, dom, fma2(mdtkap, mul2(ue, a1), pn0));
    pn1 = fma2(mdtkap, mul2(ue, a0), pn1);
    const P dt = mk2(C.dt, C.dt);
    g0 = fma2(dt, pn0, a0);
    g1 = fma2(dt, pn1, a1);
}
template <typename T>
__device__ __forceinline__ void site_vsum_whole(const SiteCoefs<T>& C, typename PK<T>::P d, typename PK<T>::P e,
                                                typename PK<T>::P& accd, typename PK<T>::P& acci)
{
    typedef typename PK<T>::P P;
    const P sq = mul2(d, d);
    if (C.quartic) accd = fma2(sq, sq, accd);
    else accd = fma2(d, d, accd);
    const P ue = mul2(d, e);
    acci = fma2(ue, ue, acci);
}

// Factor turning site_vsum's first sum into sum (u^beta - P'^beta)/beta.
template <typename T>
__device__ __forceinline__ T site_vsum_factor(bool quartic)
{
    return quartic ? T(0.25) : T(0.5);
}

// Scalar forms of site_vsum for the sums passes that run without a step: the
// potential sums of the fields as stored, about the current homogeneous mode P.
template <typename T>
__device__ __forceinline__ T vdiff_dom(T d, T P, T P2, bool quartic)
{
    const T u = d + P;
    return quartic ? (d * (u + P)) * (u * u + P2) : d * (u + P);
}
template <typename T>
__device__ __forceinline__ T vint(T d, T e, T P)
{
    const T ue = (d + P) * e;
    return ue * ue;
}

} // namespace lat
