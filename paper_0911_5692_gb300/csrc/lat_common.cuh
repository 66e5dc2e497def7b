// lat_common.cuh -- device-side state shared by the lattice kernels: the
// per-lattice constants, the FP64 scalar block that carries a(t) and the
// field-equation coefficients from one step to the next, the deterministic
// block reduction and the scale-factor update of Sec. II.B, eq. scale.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/lattice.h"

namespace lat {

// Constants of one lattice, fixed at creation (program units, Sec. II.B).
struct Model {
    int n;
    int expansion;      // 0: static; 1: eq. scale; 2: the L = 1/H form (lat_lform.cu)
    int beta;           // 2 or 4: exponent of the dominant potential term
    int stencil;        // Laplacian: 7-point or 27-point (Sec. II.C)
    int split;          // 1: phi stored as FP64 homogeneous mode + fluctuation arrays
    double dx, dt, inv_dx2;
    // factor turning the stencil's integer-weight neighbour sums into the
    // Laplacian and the gradient average: 1/dx^2 (7-point, weights 1) or
    // 1/(30 dx^2) (27-point, weights 14, 3, 1 for face, edge, corner)
    double lap_scale;
    double A, B, r, s;
    double cdom0, pdom; // V_pr dominant term: cdom0 a^pdom f^beta / beta
    double kappa0, pint;// V_pr interaction: kappa0 a^pint f^2 chi^2 / 2
    double eight_pi_G;
    double g8A2;        // eight_pi_G / A^2 (eq. scale)
    double inv_sites;   // 1 / N^3
};

// Step coefficients (DevScalars::kd, kf): the kick and drift of eq. scalar-evo
// and eq. evo, and the homogeneous inflaton mode the stored phi arrays are
// measured from (zero unless the lattice stores phi split, see below).
enum {
    kDtCl = 0,   // dt cL / dx^2 (times the stencil's 1/30 for 27 points)
    kDtCf,       // dt cF
    kMDtCdom,    // -dt cdom
    kMDtKap,     // -dt kappa
    kDt,         // dt
    kBg,         // P: homogeneous phi at the field time of the step
    kBg2,        // P^2
    kBgNew,      // P': homogeneous phi at the field time after the step
    kBgNew2,     // P'^2
    kCoefs = 10
};

// FP64 scalars that live on the device between steps. The step kernel reads the
// coefficients at its start and its last block writes those of the next step,
// so a captured CUDA graph of any number of steps needs no host round trip.
//
// Split storage of the inflaton (lat_params.split). phi = P + d with the
// homogeneous mode P (field time) and its momentum Pi (momentum time) kept here
// in FP64, and the arrays of field 0 holding the fluctuation d and its momentum.
// The homogeneous mode follows the same leapfrog with the homogeneous force,
// Pi_{n+1} = Pi_n + dt (cF P - cdom P^(beta-1)), P_{n+3/2} = P + dt Pi_{n+1}, and
// the kernels apply to d the rest of the force exactly:
//   cL Lap d + cF d - [cdom ((P+d)^(beta-1) - P^(beta-1)) + kappa (P+d) chi^2]
// for phi and -kappa (P+d)^2 chi for chi (the homogeneous value of chi stays
// zero: chi is stored whole), written without differences of nearby numbers
// (u = P + d; (u^3 - P^3) = d (u (u + P) + P^2)). The sum of the two parts is
// the same leapfrog step as for phi stored whole, so the scheme is unchanged;
// FP32 arrays then resolve the fluctuations of phi to FP32 precision of their
// own size rather than of phi. P = Pi = 0 is phi stored whole.
struct DevScalars {
    double t;        // program time of the momenta
    double a;        // scale factor at the field time t + dt/2
    double ad;       // a' at t
    double ad_next;  // a' at t + dt, solved from the sums at the field time
    double ad_half;  // a' at the field time, (ad + ad_next)/2
    double add;      // a'' at the field time (eq. scale)
    double S[4];     // <|grad f0|^2>, <|grad f1|^2>, <f0^beta/beta>, <f0^2 f1^2/2>
    double cL, cF;   // a^(-2s-2) and r(s-r+2) h^2 + r a''/a (eq. scalar-evo)
    double cdom, kappa; // potential coefficients at the field time
    long long step;  // parity of the ping-pong buffers = step & 1
    int status;      // sticky lat_status raised on the device
    unsigned int ticket; // last-block counter of the step kernel
    unsigned int ticket2;
    int pad;
    double kd[kCoefs]; // step coefficients (enum above)
    float kf[kCoefs];  // the same rounded once to FP32 for the FP32 kernels
    // History of the scalar blocks (the reverse-mode derivative's forward pass):
    // when set, the last block of each step also stores the block it produces,
    // the one the next step starts from, at log[step - log_base]. Null otherwise.
    DevScalars* log;
    long long log_base;
    // The L = 1/H form (expansion 2): the Hubble length l = a/a' of program time
    // at t, and l at t + dt as solved for the next step (lat_lform.cu).
    double ell, ell_next;
    // Homogeneous inflaton mode of split storage: P at the field time, Pi at the
    // momentum time, and both after the step being taken (zero when phi is
    // stored whole).
    double bgf, bgp, bgf_next, bgp_next;
};

// Step coefficient i for element type T (kd / kf above).
template <typename T>
__device__ __forceinline__ T step_coef(const DevScalars* sc, int i);
template <>
__device__ __forceinline__ float step_coef<float>(const DevScalars* sc, int i) { return sc->kf[i]; }
template <>
__device__ __forceinline__ double step_coef<double>(const DevScalars* sc, int i) { return sc->kd[i]; }

// Number of sums reduced per block: grad^2 of each field (unscaled by 1/dx^2),
// sum f0^beta/beta, sum f0^2 f1^2 / 2.
constexpr int kSums = 4;

// Deterministic reduction of kSums doubles over a block (any block shape; warps
// and lanes follow the linear thread index): a fixed shuffle tree within warps,
// then warp 0 folds the warp totals in warp order. Result valid in thread 0.
// `red` must hold 32 * kSums doubles.
__device__ __forceinline__ int linear_tid()
{
    return threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
}
__device__ __forceinline__ int block_warps() { return (blockDim.x * blockDim.y * blockDim.z + 31) >> 5; }

__device__ __forceinline__ void block_reduce(double v[kSums], double* red)
{
    const int tid = linear_tid(), lane = tid & 31, warp = tid >> 5;
    const int nwarps = block_warps();
#pragma unroll
    for (int k = 0; k < kSums; k++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0)
        for (int k = 0; k < kSums; k++) red[warp * kSums + k] = v[k];
    __syncthreads();
    if (warp == 0) {
        for (int k = 0; k < kSums; k++) v[k] = lane < nwarps ? red[lane * kSums + k] : 0.0;
#pragma unroll
        for (int k = 0; k < kSums; k++)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    }
    __syncthreads();
}

// Block reduction of FP32 per-thread sums: a fixed FP32 shuffle tree within
// each warp (32 terms, relative rounding error a few FP32 ulp, far below that
// of the per-thread accumulations), then warp 0 folds the warp totals in FP64 in
// warp order. FP64 arithmetic runs at a small fraction of the FP32 rate, so
// only one warp of the block touches it. Result in out[] of thread 0.
__device__ __forceinline__ void block_reduce(float v[kSums], double* red, double out[kSums])
{
    const int tid = linear_tid(), lane = tid & 31, warp = tid >> 5;
    const int nwarps = block_warps();
#pragma unroll
    for (int k = 0; k < kSums; k++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < kSums; k++) red[warp * kSums + k] = (double)v[k];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int k = 0; k < kSums; k++) {
            double w = lane < nwarps ? red[lane * kSums + k] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
            out[k] = w;
        }
    }
}

// FP64 per-thread sums: block_reduce above in FP64 throughout.
__device__ __forceinline__ void block_reduce(double v[kSums], double* red, double out[kSums])
{
    block_reduce(v, red);
#pragma unroll
    for (int k = 0; k < kSums; k++) out[k] = v[k];
}

// a^p. The exponents of the two models' rescalings (Sec. II.B) are integers
// for which repeated multiplication of a (or of inv_a = 1/a for negative p) is
// exact to a few ulp and costs a handful of FP64 multiplies instead of a
// general pow, or a division, on the slow FP64 pipe.
__device__ inline double apow(double a, double inv_a, double p)
{
    if (p == rint(p) && fabs(p) <= 16.0) {
        int e = (int)fabs(p);
        double r = 1.0, b = p < 0.0 ? inv_a : a;
        while (e) {
            if (e & 1) r *= b;
            b *= b;
            e >>= 1;
        }
        return r;
    }
    return pow(a, p);
}

// <f0^beta>/beta of the homogeneous mode alone: the potential sums of split
// storage hold the rest, sum over sites of ((P+d)^beta - P^beta)/beta.
__host__ __device__ inline double bg_potential(int beta, double P)
{
    const double q = P * P;
    return beta == 4 ? 0.25 * q * q : 0.5 * q;
}

// The per-step coefficients of eq. scalar-evo as the step kernels use them, and
// one leapfrog step of the homogeneous inflaton mode under the same cL, cF,
// cdom (its force is that of the potential at (P, chi = 0)).
__device__ inline void step_coefficients(const Model& M, DevScalars* sc)
{
    const double P = sc->bgf;
    const double force = sc->cdom * (M.beta == 4 ? P * P * P : P);
    sc->bgp_next = sc->bgp + M.dt * (sc->cF * P - force);
    sc->bgf_next = P + M.dt * sc->bgp_next;
    sc->kd[kDtCl] = M.dt * sc->cL * M.lap_scale;
    sc->kd[kDtCf] = M.dt * sc->cF;
    sc->kd[kMDtCdom] = -M.dt * sc->cdom;
    sc->kd[kMDtKap] = -M.dt * sc->kappa;
    sc->kd[kDt] = M.dt;
    sc->kd[kBg] = P;
    sc->kd[kBg2] = P * P;
    sc->kd[kBgNew] = sc->bgf_next;
    sc->kd[kBgNew2] = sc->bgf_next * sc->bgf_next;
    for (int i = 0; i < kCoefs; i++) sc->kf[i] = (float)sc->kd[i];
}

// Scale-factor update of Sec. II.B, eq. scale, with the staggered a':
// a''_{n+1/2} = q a'_{n+1/2}^2 + c, q = -(s+2)/a, a'_{n+1/2} = (a'_n + a'_{n+1})/2,
// c = (8piG/A^2) a^(-2s-2r-1) ((S0+S1)/3 + a^(2s+2) <V_pr>).
// With y = a'_n + a'_{n+1} the implicit update a'_{n+1} = a'_n + dt a''_{n+1/2}
// is (dt q/4) y^2 - y + (2a'_n + dt c) = 0; the root continuous with dt -> 0 is
// y = 2 gamma / (1 + sqrt(1 - 4 alpha gamma)). Then the coefficients of the
// field equation at the field time (eq. scalar-evo, with the f coefficient
// r(s-r+2) h^2 + r a''/a that follows from eq. fe under the rescaling).
__device__ inline void scale_solve(const Model& M, DevScalars* sc)
{
    // one FP64 division (1/a) serves every negative power and quotient below
    const double a = sc->a, ia = 1.0 / a;
    sc->cdom = M.cdom0 * apow(a, ia, M.pdom);
    sc->kappa = M.kappa0 * apow(a, ia, M.pint);
    if (!M.expansion) {
        sc->ad_next = 0.0; sc->ad_half = 0.0; sc->add = 0.0;
        sc->cL = 1.0; sc->cF = 0.0;
        step_coefficients(M, sc);
        return;
    }
    const double vpr = sc->cdom * sc->S[2] + sc->kappa * sc->S[3];
    const double c = M.g8A2 * apow(a, ia, -2.0 * M.s - 2.0 * M.r - 1.0)
                   * ((sc->S[0] + sc->S[1]) * (1.0 / 3.0) + apow(a, ia, 2.0 * M.s + 2.0) * vpr);
    const double q = -(M.s + 2.0) * ia;
    const double alpha = M.dt * q * 0.25;
    const double gamma = 2.0 * sc->ad + M.dt * c;
    const double disc = 1.0 - 4.0 * alpha * gamma;
    if (!(disc >= 0.0) || !isfinite(c)) {
        sc->status = LAT_ENONFINITE;
        return;
    }
    const double y = 2.0 * gamma / (1.0 + sqrt(disc));
    sc->ad_half = 0.5 * y;
    sc->ad_next = y - sc->ad;
    sc->add = q * sc->ad_half * sc->ad_half + c;
    sc->cL = apow(a, ia, -2.0 * M.s - 2.0);
    const double h = sc->ad_half * ia;
    sc->cF = M.r * (M.s - M.r + 2.0) * h * h + M.r * sc->add * ia;
    step_coefficients(M, sc);
}

// The scalars after one step, from those before it and the volume sums S of the
// new fields: a_{n+3/2} = a_{n+1/2} + dt a'_{n+1}, a' <- a'_{n+1}, t += dt, then
// the a' solve and coefficients for the next step (scale_solve). `advance` is
// false for the sums-only pass after initialisation or a state upload. In the
// L = 1/H form the solve for the next step is a pass of its own (its sums need
// the Laplacian of the new fields), launched after this one.
__device__ inline void advance_scalars(const Model& M, DevScalars& s, const double S[kSums], bool advance)
{
    bool finite = true;
    if (advance) {
        if (M.expansion) {
            s.a = s.a + M.dt * s.ad_next;
            s.ad = s.ad_next;
            s.ell = s.ell_next;
        }
        s.bgf = s.bgf_next;
        s.bgp = s.bgp_next;
        s.t = s.t + M.dt;
        s.step = s.step + 1;
    }
    for (int k = 0; k < kSums; k++) {
        finite = finite && isfinite(S[k]);
        s.S[k] = S[k];
    }
    // the potential sums of the kernels are taken about the homogeneous mode
    s.S[2] += bg_potential(M.beta, s.bgf);
    if (!finite) s.status = LAT_ENONFINITE;
    else if (M.expansion != 2) scale_solve(M, &s);
}

// Fixed-order reduction of the per-block partials by warp 0 of the block that
// finished last (lane l folds blocks l, l+32, ..., then a fixed shuffle tree);
// writes the averages at the new field time into out[] of thread 0.
__device__ inline void reduce_partials(const Model& M, const double* partials, int nblocks, double out[kSums])
{
    const int tid = linear_tid();
    if (tid >= 32) return;
    double v[kSums] = {0.0, 0.0, 0.0, 0.0};
    // blocks tid, tid + 32, ... in order; four of them per pass so that their
    // L2 loads are in flight together
    const double2* p2 = reinterpret_cast<const double2*>(partials);   // kSums = 4 doubles per block
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
            v[0] += x[j][0].x;
            v[1] += x[j][0].y;
            v[2] += x[j][1].x;
            v[3] += x[j][1].y;
        }
    }
    for (; b < nblocks; b += 32) {
        const double2 x0 = __ldcg(p2 + (size_t)b * 2), x1 = __ldcg(p2 + (size_t)b * 2 + 1);
        v[0] += x0.x;
        v[1] += x0.y;
        v[2] += x1.x;
        v[3] += x1.y;
    }
#pragma unroll
    for (int k = 0; k < kSums; k++)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (tid == 0) {
        out[0] = v[0] * M.lap_scale * M.inv_sites;
        out[1] = v[1] * M.lap_scale * M.inv_sites;
        out[2] = v[2] * M.inv_sites;
        out[3] = v[3] * M.inv_sites;
    }
}

// Write this block's partial sums, and let the last block of the launch fold
// all partials and advance the FP64 scalars: a_{n+3/2} = a_{n+1/2} + dt a'_{n+1},
// then the a' solve and coefficients for the next step. `advance` is false for
// the sums-only pass that follows initialisation or a state upload. The
// per-thread sums are float (FP32 kernels) or double.
template <typename A>
__device__ inline void finish_block(const Model& M, DevScalars* sc, double* partials, A v[kSums],
                                    double* red, bool advance)
{
    const int nblocks = gridDim.x * gridDim.y * gridDim.z;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const int tid = linear_tid();
    double bs[kSums];
    block_reduce(v, red, bs);
    __shared__ unsigned int is_last;
    if (tid == 0) {
        for (int k = 0; k < kSums; k++) partials[(size_t)bid * kSums + k] = bs[k];
        __threadfence();
        unsigned int t = atomicAdd(&sc->ticket, 1u);
        is_last = (t == (unsigned int)nblocks - 1u);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double S[kSums];
    reduce_partials(M, partials, nblocks, S);
    if (tid == 0) {
        // every other block has taken its ticket: the whole block can be rewritten
        DevScalars s = *sc;
        s.ticket = 0u;
        advance_scalars(M, s, S, advance);
        *sc = s;
        if (advance && s.log) s.log[s.step - s.log_base] = s;
        __threadfence();
    }
}

// As finish_block, for a domain that is part of a larger lattice (a z-slab):
// the last block writes the domain's share of the volume averages (sums over
// its sites / N^3) to sums_out and leaves the scalars alone; the scalars advance
// once the shares of every domain are added (advance_scalars).
template <typename A>
__device__ inline void finish_block_sums(const Model& M, DevScalars* sc, double* partials, A v[kSums], double* red,
                                         double* sums_out)
{
    const int nblocks = gridDim.x * gridDim.y * gridDim.z;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const int tid = linear_tid();
    double bs[kSums];
    block_reduce(v, red, bs);
    __shared__ unsigned int is_last_s;
    if (tid == 0) {
        for (int k = 0; k < kSums; k++) partials[(size_t)bid * kSums + k] = bs[k];
        __threadfence();
        is_last_s = atomicAdd(&sc->ticket, 1u) == (unsigned int)nblocks - 1u;
    }
    __syncthreads();
    if (!is_last_s) return;
    __threadfence();
    double S[kSums];
    reduce_partials(M, partials, nblocks, S);
    if (tid == 0) {
        sc->ticket = 0u;
        for (int k = 0; k < kSums; k++) sums_out[k] = S[k];
        __threadfence();
    }
}

} // namespace lat
