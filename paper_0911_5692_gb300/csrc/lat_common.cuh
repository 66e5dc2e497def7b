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
    int expansion;
    int beta;           // 2 or 4: exponent of the dominant potential term
    int pad;
    double dx, dt, inv_dx2;
    double A, B, r, s;
    double cdom0, pdom; // V_pr dominant term: cdom0 a^pdom f^beta / beta
    double kappa0, pint;// V_pr interaction: kappa0 a^pint f^2 chi^2 / 2
    double eight_pi_G;
    double inv_sites;   // 1 / N^3
};

// FP64 scalars that live on the device between steps. The step kernel reads the
// coefficients at its start and its last block writes those of the next step,
// so a captured CUDA graph of any number of steps needs no host round trip.
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
};

// Number of sums reduced per block: grad^2 of each field (unscaled by 1/dx^2),
// sum f0^beta/beta, sum f0^2 f1^2 / 2.
constexpr int kSums = 4;

// Deterministic reduction of kSums doubles over a block: a fixed shuffle tree
// within warps, then warp 0 folds the warp totals in warp order. Result valid in
// thread 0. `red` must hold 32 * kSums doubles.
__device__ __forceinline__ void block_reduce(double v[kSums], double* red)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
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
    const double a = sc->a;
    sc->cdom = M.cdom0 * pow(a, M.pdom);
    sc->kappa = M.kappa0 * pow(a, M.pint);
    if (!M.expansion) {
        sc->ad_next = 0.0; sc->ad_half = 0.0; sc->add = 0.0;
        sc->cL = 1.0; sc->cF = 0.0;
        return;
    }
    const double vpr = sc->cdom * sc->S[2] + sc->kappa * sc->S[3];
    const double c = M.eight_pi_G / (M.A * M.A) * pow(a, -2.0 * M.s - 2.0 * M.r - 1.0)
                   * ((sc->S[0] + sc->S[1]) / 3.0 + pow(a, 2.0 * M.s + 2.0) * vpr);
    const double q = -(M.s + 2.0) / a;
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
    sc->cL = pow(a, -2.0 * M.s - 2.0);
    const double h = sc->ad_half / a;
    sc->cF = M.r * (M.s - M.r + 2.0) * h * h + M.r * sc->add / a;
}

// Fixed-order reduction of the per-block partials by the block that finished
// last; writes the averages at the new field time into sc->S.
__device__ inline void reduce_partials(const Model& M, const double* partials, int nblocks, double* red,
                                       double out[kSums])
{
    double v[kSums] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < kSums; k++) v[k] += __ldcg(partials + (size_t)b * kSums + k);
    block_reduce(v, red);
    if (threadIdx.x == 0) {
        out[0] = v[0] * M.inv_dx2 * M.inv_sites;
        out[1] = v[1] * M.inv_dx2 * M.inv_sites;
        out[2] = v[2] * M.inv_sites;
        out[3] = v[3] * M.inv_sites;
    }
}

// Write this block's partial sums, and let the last block of the launch fold
// all partials and advance the FP64 scalars: a_{n+3/2} = a_{n+1/2} + dt a'_{n+1},
// then the a' solve and coefficients for the next step. `advance` is false for
// the sums-only pass that follows initialisation or a state upload.
__device__ inline void finish_block(const Model& M, DevScalars* sc, double* partials, double v[kSums],
                                    double* red, bool advance)
{
    const int nblocks = gridDim.x * gridDim.y * gridDim.z;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    block_reduce(v, red);
    __shared__ unsigned int is_last;
    if (threadIdx.x == 0) {
        for (int k = 0; k < kSums; k++) partials[(size_t)bid * kSums + k] = v[k];
        __threadfence();
        unsigned int t = atomicAdd(&sc->ticket, 1u);
        is_last = (t == (unsigned int)nblocks - 1u);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double S[kSums];
    reduce_partials(M, partials, nblocks, red, S);
    if (threadIdx.x == 0) {
        sc->ticket = 0u;
        bool finite = true;
        for (int k = 0; k < kSums; k++) finite = finite && isfinite(S[k]);
        for (int k = 0; k < kSums; k++) sc->S[k] = S[k];
        if (advance) {
            if (M.expansion) {
                sc->a = sc->a + M.dt * sc->ad_next;
                sc->ad = sc->ad_next;
            }
            sc->t = sc->t + M.dt;
            sc->step = sc->step + 1;
        }
        if (!finite) sc->status = LAT_ENONFINITE;
        else scale_solve(M, sc);
        __threadfence();
    }
}

} // namespace lat
