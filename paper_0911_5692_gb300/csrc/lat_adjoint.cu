// lat_adjoint.cu -- reverse-mode derivative of the leapfrog evolution (the
// adjoint of Sec. II.B, eq. evo with eq. scalar-evo and eq. scale), with
// sqrt(n) checkpointing and recomputation.
//
// Forward step k (state f_k, pi_k, a_k, a'_k; volume sums S_k of f_k):
//   a'' and the coefficients cL, cF, cdom, kappa from (a_k, a'_k, S_k) (the
//   implicit a' update of eq. scale, solved as a quadratic in y = a'_k + a'_{k+1})
//   pi_{k+1} = pi_k + dt (cL Lap f_k + cF f_k - dV/df(f_k))
//   f_{k+1}  = f_k + dt pi_{k+1},  a'_{k+1} = y - a'_k,  a_{k+1} = a_k + dt a'_{k+1}
// Reverse step k, from the adjoint (fb, pb) of (f_{k+1}, pi_{k+1}):
//   pt = pb + dt fb                                  (drift)
//   fb_k = fb + dt (cL Lap pt + cF pt - Hess V(f_k) pt) + sum_j Sb_j dS_j/df(f_k)
//   pb_k = pt
// where Sb, the adjoint of the volume sums S_k, comes from the FP64 reverse of
// the scalar update, whose inputs are four volume sums of pt against f_k:
//   dt <pt, Lap f_k>, dt <pt, f_k>, -dt <pt0, f0^(beta-1)>, -dt <pt0 f0 f1^2 + pt1 f0^2 f1>.
// One kernel per reverse step does the field update of step k and, from the
// pt it has just formed, the four sums of step k-1; its last block runs the
// scalar reverse of step k-1. Memory traffic per reverse step: read f_k,
// f_{k-1} and the incoming adjoints, write the outgoing adjoints.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <type_traits>
#include <vector>

#include "lat_async.cuh"
#include "lat_internal.h"
#include "lat_pairs.cuh"

namespace lat {

namespace {

constexpr int kAdjThreads = 256;

// Adjoint scalars carried between reverse steps (FP64, device).
struct AdjScalars {
    double ba, bad, bk0;     // adjoints of a, a' of the state being reached, and of kappa0
    double cL, cF, cd, kp;   // forward coefficients of the step the next field update reverses
    double bS[4];            // adjoint of that step's volume sums
    int status;
    unsigned int ticket;
};

template <typename T>
struct AdjBufs {
    const T* f[2];    // f_k, the fields the reversed step started from
    const T* fm[2];   // f_{k-1}, or null when there is no earlier step
    const T* fb[2];   // adjoint of f_{k+1}
    const T* pb[2];   // adjoint of pi_{k+1}
    T* fbo[2];        // adjoint of f_k (out)
    T* pbo[2];        // adjoint of pi_k (out)
};

// Intermediate values of the forward scalar update of one step.
struct ScaleFwd {
    double c, q, alpha, y, ah, add, vpr, ea, eb;
};

// Recompute the forward scalar update from the scalars the step started from
// (same formulas as scale_solve, with the intermediates kept). ia = 1/a.
__device__ void scale_forward(const Model& M, const DevScalars& s, double ia, ScaleFwd& o)
{
    const double a = s.a;
    o.vpr = s.cdom * s.S[2] + s.kappa * s.S[3];
    o.ea = apow(a, ia, -2.0 * M.s - 2.0 * M.r - 1.0);
    o.eb = apow(a, ia, 2.0 * M.s + 2.0);
    o.c = M.g8A2 * o.ea * ((s.S[0] + s.S[1]) * (1.0 / 3.0) + o.eb * o.vpr);
    o.q = -(M.s + 2.0) * ia;
    o.alpha = M.dt * o.q * 0.25;
    o.y = 2.0 * s.ad_half;
    o.ah = s.ad_half;
    o.add = s.add;
}

// Reverse of the scalar update of one step: given the adjoints of the
// coefficients the kick used (bcL, bcF, bcd, bkp) and of y (from the a, a'
// update), add to the adjoints of a, a' and kappa0 (ba, bad, bk0, kept in
// registers by the caller) and produce those of S. One reciprocal of a and one
// of the solve's denominator serve every quotient (the FP64 pipe is narrow and
// this runs in one thread).
__device__ void scale_reverse(const Model& M, const DevScalars& s, double bcL, double bcF, double bcd, double bkp,
                              double by, double& ba_io, double& bad_io, double& bk0_io, double bS[4])
{
    const double a = s.a, ia = 1.0 / a, ia2 = ia * ia;
    double ba = 0.0, bad = 0.0;
    for (int k = 0; k < 4; k++) bS[k] = 0.0;
    if (M.expansion) {
        ScaleFwd o;
        scale_forward(M, s, ia, o);
        const double r = M.r, sx = M.s;
        const double hh = o.ah * ia;
        // cF = r(s-r+2) h^2 + r a''/a, h = a'_half / a
        const double bh = bcF * 2.0 * r * (sx - r + 2.0) * hh;
        const double badd = bcF * r * ia;
        ba -= bcF * r * o.add * ia2;
        double bah = bh * ia;
        ba -= bh * o.ah * ia2;
        // a'' = q a'_half^2 + c
        double bq = badd * o.ah * o.ah;
        bah += badd * 2.0 * o.q * o.ah;
        double bc = badd;
        // a'_half = y / 2; y solves alpha y^2 - y + gamma = 0 with gamma = 2a' + dt c
        by += 0.5 * bah;
        const double iden = 1.0 / (1.0 - 2.0 * o.alpha * o.y);
        const double bgamma = by * iden, balpha = by * o.y * o.y * iden;
        bq += balpha * M.dt * 0.25;
        bad += 2.0 * bgamma;
        bc += M.dt * bgamma;
        ba += bq * (sx + 2.0) * ia2;
        // cL = a^(-2s-2)
        ba += bcL * (-2.0 * sx - 2.0) * apow(a, ia, -2.0 * sx - 3.0);
        // c = K ea (T + eb vpr)
        const double K = M.g8A2;
        const double T = (s.S[0] + s.S[1]) * (1.0 / 3.0);
        const double bea = bc * K * (T + o.eb * o.vpr);
        const double bT = bc * K * o.ea;
        const double beb = bc * K * o.ea * o.vpr;
        const double bvpr = bc * K * o.ea * o.eb;
        ba += bea * (-2.0 * sx - 2.0 * r - 1.0) * apow(a, ia, -2.0 * sx - 2.0 * r - 2.0);
        ba += beb * (2.0 * sx + 2.0) * apow(a, ia, 2.0 * sx + 1.0);
        bS[0] = bT * (1.0 / 3.0);
        bS[1] = bT * (1.0 / 3.0);
        bcd += bvpr * s.S[2];
        bkp += bvpr * s.S[3];
        bS[2] = bvpr * s.cdom;
        bS[3] = bvpr * s.kappa;
    }
    // cdom = cdom0 a^pdom, kappa = kappa0 a^pint
    ba += bcd * M.cdom0 * M.pdom * apow(a, ia, M.pdom - 1.0) + bkp * M.kappa0 * M.pint * apow(a, ia, M.pint - 1.0);
    bk0_io += bkp * apow(a, ia, M.pint);
    ba_io += ba;
    bad_io += bad;
}

template <typename T>
__device__ __forceinline__ T powb1(T f, int beta)   // f^(beta-1), beta in {2, 4}
{
    return beta == 4 ? f * f * f : f;
}

// Fold the per-thread sums of a reverse-step kernel (block reduction, then the
// last block of the launch in fixed order) and run the FP64 scalar reverse of
// step k-1 from them; hist = the scalars step k-1 started from. Writes the
// coefficients and the adjoint of the sums that the next field update uses.
template <typename T>
__device__ void adj_finish(T acc[kSums], double* red, AdjScalars* as, const DevScalars* hist, double* partials,
                           const Model& M)
{
    double bs[kSums];
    block_reduce(acc, red, bs);
    __shared__ unsigned int is_last;
    const int nblocks = gridDim.x * gridDim.y * gridDim.z;
    const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
    if (tid == 0) {
        for (int k = 0; k < kSums; k++) partials[(size_t)bid * kSums + k] = bs[k];
        __threadfence();
        is_last = atomicAdd(&as->ticket, 1u) == (unsigned int)nblocks - 1u;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    if (tid >= 32) return;
    double v[kSums] = {0.0, 0.0, 0.0, 0.0};
    // blocks tid, tid + 32, ... in order, four per pass so that their L2 loads
    // are in flight together
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
    if (tid != 0) return;
    // the scalar adjoints live in registers for the serial FP64 part
    double ba = as->ba, bad = as->bad, bk0 = as->bk0;
    as->ticket = 0u;
    const DevScalars s = *hist;
    // reverse of a_{k} = a_{k-1} + dt a'_{k}, a'_{k} = y - a'_{k-1}
    double by = 0.0;
    if (M.expansion) {
        by = bad + M.dt * ba;
        bad = -by;
    }
    const double bcL = M.dt * v[0] * M.inv_dx2, bcF = M.dt * v[1], bcd = -M.dt * v[2], bkp = -M.dt * v[3];
    double bS[4];
    scale_reverse(M, s, bcL, bcF, bcd, bkp, by, ba, bad, bk0, bS);
    bool finite = isfinite(ba) && isfinite(bad) && isfinite(bk0);
    for (int k = 0; k < 4; k++) {
        as->bS[k] = bS[k];
        finite = finite && isfinite(bS[k]);
    }
    as->ba = ba;
    as->bad = bad;
    as->bk0 = bk0;
    as->cL = s.cL;
    as->cF = s.cF;
    as->cd = s.cdom;
    as->kp = s.kappa;
    if (!finite) as->status = LAT_ENONFINITE;
    __threadfence();
}

// Reverse step kernel, one site per thread (any N). UPDATE: reverse the field update of step k (outputs fbo,
// pbo); always: if fm is given, the four sums of step k-1 from pt' = pb_k + dt fb_k
// (without UPDATE, pb + dt fb of the inputs), folded by the last block into the
// scalar reverse of step k-1 (hist = the scalars step k-1 started from).
template <typename T, bool UPDATE>
__global__ void __launch_bounds__(kAdjThreads) adj_step_kernel(AdjBufs<T> B, Model M, AdjScalars* as,
                                                               const DevScalars* hist, double* partials)
{
    __shared__ double red[32 * kSums];
    if (as->status != LAT_OK) return;
    const int n = M.n;
    const long long nn = (long long)n * n, n3 = nn * n;
    const T dt = (T)M.dt;
    const T cLs = (T)(as->cL * M.inv_dx2), cF = (T)as->cF, cd = (T)as->cd, kp = (T)as->kp;
    const T sg0 = (T)(-2.0 * as->bS[0] * M.inv_dx2 * M.inv_sites), sg1 = (T)(-2.0 * as->bS[1] * M.inv_dx2 * M.inv_sites);
    const T sv2 = (T)(as->bS[2] * M.inv_sites), sv3 = (T)(as->bS[3] * M.inv_sites);
    const int beta = M.beta;
    const bool sums = B.fm[0] != nullptr;
    T acc[kSums] = {T(0), T(0), T(0), T(0)};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % n), y = (int)((i / n) % n), z = (int)(i / nn);
        const long long ixm = i + ((x == 0 ? n - 1 : x - 1) - x), ixp = i + ((x == n - 1 ? 0 : x + 1) - x);
        const long long iym = i + (long long)((y == 0 ? n - 1 : y - 1) - y) * n;
        const long long iyp = i + (long long)((y == n - 1 ? 0 : y + 1) - y) * n;
        const long long izm = i + ((z == 0 ? n - 1 : z - 1) - z) * nn;
        const long long izp = i + ((z == n - 1 ? 0 : z + 1) - z) * nn;
        T ptn[2];   // pt' of step k-1 at this site
        if (UPDATE) {
            T pt[2], lpt[2], lf[2];
#pragma unroll
            for (int f = 0; f < 2; f++) {
                const T* pb = B.pb[f];
                const T* fb = B.fb[f];
                const T c = __ldg(pb + i) + dt * __ldg(fb + i);
                pt[f] = c;
                lpt[f] = ((__ldg(pb + ixm) + dt * __ldg(fb + ixm)) - c) + ((__ldg(pb + ixp) + dt * __ldg(fb + ixp)) - c) +
                         ((__ldg(pb + iym) + dt * __ldg(fb + iym)) - c) + ((__ldg(pb + iyp) + dt * __ldg(fb + iyp)) - c) +
                         ((__ldg(pb + izm) + dt * __ldg(fb + izm)) - c) + ((__ldg(pb + izp) + dt * __ldg(fb + izp)) - c);
                const T* ff = B.f[f];
                const T fc = __ldg(ff + i);
                lf[f] = (__ldg(ff + ixm) - fc) + (__ldg(ff + ixp) - fc) + (__ldg(ff + iym) - fc) + (__ldg(ff + iyp) - fc) +
                        (__ldg(ff + izm) - fc) + (__ldg(ff + izp) - fc);
            }
            const T f0 = __ldg(B.f[0] + i), f1 = __ldg(B.f[1] + i);
            // Hessian of V_pr = cdom f0^beta/beta + kappa f0^2 f1^2/2
            const T h00 = (beta == 4 ? T(3) * cd * f0 * f0 : cd) + kp * f1 * f1;
            const T h01 = T(2) * kp * f0 * f1;
            const T h11 = kp * f0 * f0;
            const T g0 = cLs * lpt[0] + cF * pt[0] - h00 * pt[0] - h01 * pt[1];
            const T g1 = cLs * lpt[1] + cF * pt[1] - h01 * pt[0] - h11 * pt[1];
            const T s0 = sg0 * lf[0] + sv2 * powb1(f0, beta) + sv3 * f0 * f1 * f1;
            const T s1 = sg1 * lf[1] + sv3 * f0 * f0 * f1;
            const T nf0 = __ldg(B.fb[0] + i) + dt * g0 + s0;
            const T nf1 = __ldg(B.fb[1] + i) + dt * g1 + s1;
            B.fbo[0][i] = nf0;
            B.fbo[1][i] = nf1;
            B.pbo[0][i] = pt[0];
            B.pbo[1][i] = pt[1];
            ptn[0] = pt[0] + dt * nf0;
            ptn[1] = pt[1] + dt * nf1;
        } else {
            ptn[0] = __ldg(B.pb[0] + i) + dt * __ldg(B.fb[0] + i);
            ptn[1] = __ldg(B.pb[1] + i) + dt * __ldg(B.fb[1] + i);
        }
        if (sums) {
            T lm[2];
#pragma unroll
            for (int f = 0; f < 2; f++) {
                const T* ff = B.fm[f];
                const T fc = __ldg(ff + i);
                lm[f] = (__ldg(ff + ixm) - fc) + (__ldg(ff + ixp) - fc) + (__ldg(ff + iym) - fc) + (__ldg(ff + iyp) - fc) +
                        (__ldg(ff + izm) - fc) + (__ldg(ff + izp) - fc);
            }
            const T m0 = __ldg(B.fm[0] + i), m1 = __ldg(B.fm[1] + i);
            acc[0] += ptn[0] * lm[0] + ptn[1] * lm[1];
            acc[1] += ptn[0] * m0 + ptn[1] * m1;
            acc[2] += ptn[0] * powb1(m0, beta);
            acc[3] += ptn[0] * m0 * m1 * m1 + ptn[1] * m0 * m0 * m1;
        }
    }
    if (!sums) return;
    adj_finish(acc, red, as, hist, partials, M);
}

// Reverse step kernel as a z-march (N a multiple of 32): a 32 x 8 tile of
// threads walks a run of z planes; each thread keeps the z-1, z, z+1 values of
// the six stencil arrays (pt = pb + dt fb, f_k and f_{k-1} of both fields) in
// registers and takes its x and y neighbours from a shared-memory copy of the
// current plane with a one-site halo (two copies used alternately, so one
// barrier per plane suffices). Each thread stages the raw values of its own
// site for the planes two and three ahead in shared memory by asynchronous
// copies (no registers held while they are in flight, and no barrier: a thread
// reads back only what it copied); halo values are loaded one plane ahead.
// Same arithmetic as adj_step_kernel.
constexpr int kMX = 32, kMY = 8, kStage = 3;

template <typename T>
constexpr size_t adj_march_smem()
{
    return sizeof(T) * ((size_t)kStage * 8 * kMX * kMY + 2 * 6 * (kMY + 2) * (kMX + 2));
}

template <typename T>
__global__ void __launch_bounds__(kMX * kMY, sizeof(T) == 4 ? 3 : 2)
    adj_march_kernel(AdjBufs<T> B, Model M, AdjScalars* as, const DevScalars* hist, double* partials, int nzc)
{
    __shared__ double red[32 * kSums];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T (*stage)[8][kMX * kMY] = reinterpret_cast<T (*)[8][kMX * kMY]>(smem_raw);
    T (*tiles)[6][kMY + 2][kMX + 2] =
        reinterpret_cast<T (*)[6][kMY + 2][kMX + 2]>(smem_raw + sizeof(T) * kStage * 8 * kMX * kMY);
    if (as->status != LAT_OK) return;
    const int n = M.n;
    const uint32_t nn = (uint32_t)n * n;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kMX + tx;
    const int x = blockIdx.x * kMX + tx, y = blockIdx.y * kMY + ty;
    const int z0 = (int)((long long)blockIdx.z * n / nzc);
    const int nz = (int)((long long)(blockIdx.z + 1) * n / nzc) - z0;
    const T dt = (T)M.dt;
    const T cLs = (T)(as->cL * M.inv_dx2), cF = (T)as->cF, cd = (T)as->cd, kp = (T)as->kp;
    const T sg0 = (T)(-2.0 * as->bS[0] * M.inv_dx2 * M.inv_sites), sg1 = (T)(-2.0 * as->bS[1] * M.inv_dx2 * M.inv_sites);
    const T sv2 = (T)(as->bS[2] * M.inv_sites), sv3 = (T)(as->bS[3] * M.inv_sites);
    const int beta = M.beta;
    const bool sums = B.fm[0] != nullptr;
    // raw arrays: 0,1 pb; 2,3 fb; 4,5 f_k; 6,7 f_{k-1}
    const T* R[8] = {B.pb[0], B.pb[1], B.fb[0], B.fb[1], B.f[0], B.f[1], B.fm[0], B.fm[1]};
    const int nraw = sums ? 8 : 6;
    const uint32_t col = (uint32_t)y * n + x;
    // the one halo site this thread also fetches in x and in y (edge threads)
    const bool hx = tx == 0 || tx == kMX - 1, hy = ty == 0 || ty == kMY - 1;
    const uint32_t colx = (uint32_t)y * n + (tx == 0 ? (x == 0 ? n - 1 : x - 1) : (x == n - 1 ? 0 : x + 1));
    const uint32_t coly = (uint32_t)(ty == 0 ? (y == 0 ? n - 1 : y - 1) : (y == n - 1 ? 0 : y + 1)) * n + x;
    const int sx = tx == 0 ? 0 : kMX + 1, sy = ty == 0 ? 0 : kMY + 1;
    auto plane_of = [&](int z) -> uint32_t { return (uint32_t)(z < 0 ? z + n : (z >= n ? z - n : z)) * nn; };
    // stencil value a (0..5) from raw values
    auto st = [&](const T* r, int a) -> T { return a < 2 ? r[a] + dt * r[a + 2] : r[a + 2]; };
    // copies of this site's raw values of plane z into stage slot s
    auto stage_plane = [&](int z, int s) {
        const uint32_t o = plane_of(z) + col;
#pragma unroll
        for (int q = 0; q < 8; q++)
            if (q < nraw) cp_async_small<sizeof(T)>(&stage[s][q][tid], R[q] + o);
    };

    T w[6][3];           // stencil arrays at z-1, z, z+1
    T fbz[2][2];         // raw fb at z, z+1
    T hxr[8], hyr[8];    // raw halo values of the next plane
    {
        T r0[8], r1[8];
        const uint32_t pm = plane_of(z0 - 1) + col, pc = plane_of(z0) + col;
#pragma unroll
        for (int q = 0; q < 8; q++)
            if (q < nraw) {
                r0[q] = __ldg(R[q] + pm);
                r1[q] = __ldg(R[q] + pc);
                if (hx) hxr[q] = __ldg(R[q] + pc - col + colx);
                if (hy) hyr[q] = __ldg(R[q] + pc - col + coly);
            }
#pragma unroll
        for (int a = 0; a < 6; a++)
            if (a + 2 < nraw) {
                w[a][0] = st(r0, a);
                w[a][1] = st(r1, a);
            }
        fbz[0][0] = r1[2];
        fbz[1][0] = r1[3];
    }
    // group j (j = 0, 1) stages plane z0+1+j into slot j; plane k then stages
    // z0+k+3 into slot (k+2) % 3 after reading slot k % 3 (waiting for group k)
    stage_plane(z0 + 1, 0);
    cp_async_commit();
    if (nz > 1) stage_plane(z0 + 2, 1);
    cp_async_commit();
    T acc[kSums] = {T(0), T(0), T(0), T(0)};
    int sr = 0, sw = 2;   // k % 3, (k + 2) % 3
    for (int k = 0; k < nz; k++) {
        const int z = z0 + k;
        T(*tile)[kMY + 2][kMX + 2] = tiles[k & 1];
        cp_async_wait(1);
        T raw[8];
#pragma unroll
        for (int q = 0; q < 8; q++)
            if (q < nraw) raw[q] = stage[sr][q][tid];
        if (k + 2 < nz) stage_plane(z + 3, sw);
        cp_async_commit();
        sr = sr == 2 ? 0 : sr + 1;
        sw = sw == 2 ? 0 : sw + 1;
#pragma unroll
        for (int a = 0; a < 6; a++)
            if (a + 2 < nraw) {
                w[a][2] = st(raw, a);
                tile[a][ty + 1][tx + 1] = w[a][1];
                if (hx) tile[a][ty + 1][sx] = st(hxr, a);
                if (hy) tile[a][sy][tx + 1] = st(hyr, a);
            }
        fbz[0][1] = raw[2];
        fbz[1][1] = raw[3];
        // halo of the next plane
        if (k + 1 < nz) {
            const uint32_t p1 = plane_of(z + 1);
#pragma unroll
            for (int q = 0; q < 8; q++)
                if (q < nraw) {
                    if (hx) hxr[q] = __ldg(R[q] + p1 + colx);
                    if (hy) hyr[q] = __ldg(R[q] + p1 + coly);
                }
        }
        __syncthreads();
        T lap[6];
#pragma unroll
        for (int a = 0; a < 6; a++)
            if (a + 2 < nraw) {
                const T c = w[a][1];
                lap[a] = (tile[a][ty + 1][tx] - c) + (tile[a][ty + 1][tx + 2] - c) + (tile[a][ty][tx + 1] - c) +
                         (tile[a][ty + 2][tx + 1] - c) + (w[a][0] - c) + (w[a][2] - c);
            }
        const T pt0 = w[0][1], pt1 = w[1][1], f0 = w[2][1], f1 = w[3][1];
        const T h00 = (beta == 4 ? T(3) * cd * f0 * f0 : cd) + kp * f1 * f1;
        const T h01 = T(2) * kp * f0 * f1;
        const T h11 = kp * f0 * f0;
        const T g0 = cLs * lap[0] + cF * pt0 - h00 * pt0 - h01 * pt1;
        const T g1 = cLs * lap[1] + cF * pt1 - h01 * pt0 - h11 * pt1;
        const T s0 = sg0 * lap[2] + sv2 * powb1(f0, beta) + sv3 * f0 * f1 * f1;
        const T s1 = sg1 * lap[3] + sv3 * f0 * f0 * f1;
        const T nf0 = fbz[0][0] + dt * g0 + s0;
        const T nf1 = fbz[1][0] + dt * g1 + s1;
        const uint32_t i = (uint32_t)z * nn + col;
        B.fbo[0][i] = nf0;
        B.fbo[1][i] = nf1;
        B.pbo[0][i] = pt0;
        B.pbo[1][i] = pt1;
        if (sums) {
            const T q0 = pt0 + dt * nf0, q1 = pt1 + dt * nf1;
            const T m0 = w[4][1], m1 = w[5][1];
            acc[0] += q0 * lap[4] + q1 * lap[5];
            acc[1] += q0 * m0 + q1 * m1;
            acc[2] += q0 * powb1(m0, beta);
            acc[3] += q0 * m0 * m1 * m1 + q1 * m0 * m0 * m1;
        }
#pragma unroll
        for (int a = 0; a < 6; a++) {
            w[a][0] = w[a][1];
            w[a][1] = w[a][2];
        }
        fbz[0][0] = fbz[0][1];
        fbz[1][0] = fbz[1][1];
    }
    cp_async_wait(0);
    if (!sums) return;
    adj_finish(acc, red, as, hist, partials, M);
}

// FP32 reverse step with two x sites per thread (N a multiple of 64): the
// z-march of adj_march_kernel on a 64 x 8 site tile, with packed f32x2
// arithmetic (one instruction updates both sites) and 8-byte staged copies, so
// the per-site instruction count (addresses, loop, barriers) is halved. Each
// thread stages the raw values of its site pair for the next plane, and edge
// threads the halo values of the next plane, in shared memory by asynchronous
// copies; halos are written into the next plane's copy of the tile right after
// the current plane's barrier (that copy was last read before it).
constexpr int kPX = 32, kPY = 8, kPW = 2 * kPX + 4;   // threads in x, y; tile row (halo + 64 + halo + pad)

struct AdjPairSmem {
    F2 stage[2][8][kPX * kPY];       // raw values of each thread's site pair, by plane parity
    float sx[2][8][kPY][2];          // x-halo raw values (left of lane 0, right of lane 31)
    F2 sy[2][8][2][kPX];             // y-halo raw pairs (below warp 0, above warp kPY-1)
    float tile[2][6][kPY + 2][kPW];  // stencil values of the current plane with a one-site halo
};

__global__ void __launch_bounds__(kPX * kPY, 2)
    adj_pair_kernel(AdjBufs<float> B, Model M, AdjScalars* as, const DevScalars* hist, double* partials, int nzc)
{
    __shared__ double red[32 * kSums];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    AdjPairSmem& SM = *reinterpret_cast<AdjPairSmem*>(smem_raw);
    if (as->status != LAT_OK) return;
    const int n = M.n;
    const uint32_t nn = (uint32_t)n * n;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kPX + tx;
    const int x0 = blockIdx.x * (2 * kPX) + 2 * tx, y = blockIdx.y * kPY + ty;
    const int z0 = (int)((long long)blockIdx.z * n / nzc);
    const int nz = (int)((long long)(blockIdx.z + 1) * n / nzc) - z0;
    const float dts = (float)M.dt;
    const F2 dt = mk2(dts, dts);
    const float cLv = (float)(as->cL * M.inv_dx2);
    const F2 cLs = mk2(cLv, cLv), cF = mk2((float)as->cF, (float)as->cF);
    const F2 cd = mk2((float)as->cd, (float)as->cd), kp = mk2((float)as->kp, (float)as->kp);
    const float g0v = (float)(-2.0 * as->bS[0] * M.inv_dx2 * M.inv_sites), g1v = (float)(-2.0 * as->bS[1] * M.inv_dx2 * M.inv_sites);
    const F2 sg0 = mk2(g0v, g0v), sg1 = mk2(g1v, g1v);
    const F2 sv2 = mk2((float)(as->bS[2] * M.inv_sites), (float)(as->bS[2] * M.inv_sites));
    const F2 sv3 = mk2((float)(as->bS[3] * M.inv_sites), (float)(as->bS[3] * M.inv_sites));
    const F2 two = mk2(2.0f, 2.0f), three = mk2(3.0f, 3.0f);
    const bool quartic = M.beta == 4;
    const bool sums = B.fm[0] != nullptr;
    const float* R[8] = {B.pb[0], B.pb[1], B.fb[0], B.fb[1], B.f[0], B.f[1], B.fm[0], B.fm[1]};
    const int nraw = sums ? 8 : 6;
    const uint32_t col = (uint32_t)y * n + x0;
    const float* Rc[8];   // this thread's site pair in each array (plane 0)
#pragma unroll
    for (int q = 0; q < 8; q++) Rc[q] = q < nraw ? R[q] + col : nullptr;
    // Halo sites are fetched by warps 0 and kPY-1 only (warp-uniform branches):
    // every lane of warp 0 the pair below the tile, every lane of warp kPY-1 the
    // pair above it, and lanes 0..2kPY-1 of warp 0 the single sites left and
    // right of the tile's rows (row = lane % kPY, side = lane / kPY).
    const bool wb = ty == 0, wa = ty == kPY - 1;
    const bool xh = wb && tx < 2 * kPY;
    const int xrow = tx % kPY, xside = tx / kPY;
    const int xt = blockIdx.x * (2 * kPX), y0 = blockIdx.y * kPY;
    const uint32_t colx = (uint32_t)(y0 + xrow) * n +
                          (xside ? (xt + 2 * kPX == n ? 0 : xt + 2 * kPX) : (xt == 0 ? n - 1 : xt - 1));
    const uint32_t coly = (uint32_t)(wb ? (y0 == 0 ? n - 1 : y0 - 1) : (y0 + kPY == n ? 0 : y0 + kPY)) * n + x0;
    auto plane_of = [&](int z) -> uint32_t { return (uint32_t)(z < 0 ? z + n : (z >= n ? z - n : z)) * nn; };
    auto st2 = [&](const F2* r, int a) -> F2 { return a < 2 ? fma2(dt, r[a + 2], r[a]) : r[a + 2]; };
    auto st1 = [&](const float* r, int a) -> float { return a < 2 ? r[a] + dts * r[a + 2] : r[a + 2]; };
    // copies of plane z into stage slot s: this thread's pair, and halo sites
    auto stage_plane = [&](int z, int s) {
        const uint32_t o = plane_of(z);
#pragma unroll
        for (int q = 0; q < 8; q++)
            if (q < nraw) cp_async_small<8>(&SM.stage[s][q][tid], Rc[q] + o);
        if (wb || wa) {
#pragma unroll
            for (int q = 0; q < 8; q++)
                if (q < nraw) cp_async_small<8>(&SM.sy[s][q][wa][tx], R[q] + o + coly);
            if (xh) {
#pragma unroll
                for (int q = 0; q < 8; q++)
                    if (q < nraw) cp_async_small<4>(&SM.sx[s][q][xrow][xside], R[q] + o + colx);
            }
        }
    };
    // halos of the plane in slot s into tile t
    auto halo_to_tile = [&](int s, int t) {
        if (!(wb || wa)) return;
        {
            F2 r[8];
#pragma unroll
            for (int q = 0; q < 8; q++)
                if (q < nraw) r[q] = SM.sy[s][q][wa][tx];
#pragma unroll
            for (int a = 0; a < 6; a++)
                if (a + 2 < nraw)
                    *reinterpret_cast<F2*>(&SM.tile[t][a][wb ? 0 : kPY + 1][2 + 2 * tx]) = st2(r, a);
        }
        if (xh) {
            float r[8];
#pragma unroll
            for (int q = 0; q < 8; q++)
                if (q < nraw) r[q] = SM.sx[s][q][xrow][xside];
#pragma unroll
            for (int a = 0; a < 6; a++)
                if (a + 2 < nraw) SM.tile[t][a][xrow + 1][xside ? 2 * kPX + 2 : 1] = st1(r, a);
        }
    };

    F2 w[6][3];          // stencil pairs at z-1, z, z+1
    F2 fbz[2][2];        // raw fb pairs at z, z+1
    {
        F2 r0[8], r1[8];
        const uint32_t pm = plane_of(z0 - 1), pc = plane_of(z0);
#pragma unroll
        for (int q = 0; q < 8; q++)
            if (q < nraw) {
                r0[q] = *reinterpret_cast<const F2*>(Rc[q] + pm);
                r1[q] = *reinterpret_cast<const F2*>(Rc[q] + pc);
            }
#pragma unroll
        for (int a = 0; a < 6; a++)
            if (a + 2 < nraw) {
                w[a][0] = st2(r0, a);
                w[a][1] = st2(r1, a);
            }
        fbz[0][0] = r1[2];
        fbz[1][0] = r1[3];
    }
    // halos of plane z0 straight into tile 0; plane z0+1 staged into slot 1
    stage_plane(z0, 0);
    cp_async_commit();
    if (nz > 0) stage_plane(z0 + 1, 1);
    cp_async_commit();
    cp_async_wait(1);
    halo_to_tile(0, 0);
    F2 acc[kSums] = {mk2(0.f, 0.f), mk2(0.f, 0.f), mk2(0.f, 0.f), mk2(0.f, 0.f)};
    // plane k of the run, T_ = k & 1 as a compile-time constant (slot and
    // tile offsets fold into immediates)
    auto plane_step = [&](int k, auto T_) {
        constexpr int t = decltype(T_)::value, sn = 1 - t;
        const int z = z0 + k;
        float(*tile)[kPY + 2][kPW] = SM.tile[t];
        cp_async_wait(0);   // plane z+1 in slot sn
        F2 raw[8];
#pragma unroll
        for (int q = 0; q < 8; q++)
            if (q < nraw) raw[q] = SM.stage[sn][q][tid];
        // plane z+2 into the other slot (its plane z was read a plane ago)
        if (k + 1 < nz) stage_plane(z + 2, t);
        cp_async_commit();
#pragma unroll
        for (int a = 0; a < 6; a++)
            if (a + 2 < nraw) {
                w[a][2] = st2(raw, a);
                *reinterpret_cast<F2*>(&tile[a][ty + 1][2 + 2 * tx]) = w[a][1];
            }
        fbz[0][1] = raw[2];
        fbz[1][1] = raw[3];
        __syncthreads();
        // the next plane's halos, into the copy of the tile read before this barrier
        if (k + 1 < nz) halo_to_tile(sn, 1 - t);
        F2 lap[6];
#pragma unroll
        for (int a = 0; a < 6; a++)
            if (a + 2 < nraw) {
                const F2 c = w[a][1];
                const F2 lft = mk2(tile[a][ty + 1][1 + 2 * tx], lo2(c));
                const F2 rgt = mk2(hi2(c), tile[a][ty + 1][4 + 2 * tx]);
                const F2 up = *reinterpret_cast<const F2*>(&tile[a][ty][2 + 2 * tx]);
                const F2 dn = *reinterpret_cast<const F2*>(&tile[a][ty + 2][2 + 2 * tx]);
                lap[a] = add2(add2(add2(sub2(lft, c), sub2(rgt, c)), add2(sub2(up, c), sub2(dn, c))),
                              add2(sub2(w[a][0], c), sub2(w[a][2], c)));
            }
        const F2 pt0 = w[0][1], pt1 = w[1][1], f0 = w[2][1], f1 = w[3][1];
        const F2 f0f0 = mul2(f0, f0), f1f1 = mul2(f1, f1), f0f1 = mul2(f0, f1);
        const F2 h00 = fma2(kp, f1f1, quartic ? mul2(mul2(three, cd), f0f0) : cd);
        const F2 h01 = mul2(mul2(two, kp), f0f1);
        const F2 h11 = mul2(kp, f0f0);
        // g = cL Lap pt + cF pt - H pt
        const F2 g0 = sub2(fma2(cLs, lap[0], mul2(cF, pt0)), fma2(h00, pt0, mul2(h01, pt1)));
        const F2 g1 = sub2(fma2(cLs, lap[1], mul2(cF, pt1)), fma2(h01, pt0, mul2(h11, pt1)));
        const F2 f0b = quartic ? mul2(f0f0, f0) : f0;
        const F2 s0 = fma2(sg0, lap[2], fma2(sv2, f0b, mul2(sv3, mul2(f0, f1f1))));
        const F2 s1 = fma2(sg1, lap[3], mul2(sv3, mul2(f0f0, f1)));
        const F2 nf0 = add2(fma2(dt, g0, fbz[0][0]), s0);
        const F2 nf1 = add2(fma2(dt, g1, fbz[1][0]), s1);
        const uint32_t i = (uint32_t)z * nn + col;
        *reinterpret_cast<F2*>(B.fbo[0] + i) = nf0;
        *reinterpret_cast<F2*>(B.fbo[1] + i) = nf1;
        *reinterpret_cast<F2*>(B.pbo[0] + i) = pt0;
        *reinterpret_cast<F2*>(B.pbo[1] + i) = pt1;
        if (sums) {
            const F2 q0 = fma2(dt, nf0, pt0), q1 = fma2(dt, nf1, pt1);
            const F2 m0 = w[4][1], m1 = w[5][1];
            const F2 m0m0 = mul2(m0, m0), m1m1 = mul2(m1, m1);
            acc[0] = fma2(q0, lap[4], fma2(q1, lap[5], acc[0]));
            acc[1] = fma2(q0, m0, fma2(q1, m1, acc[1]));
            acc[2] = fma2(q0, quartic ? mul2(m0m0, m0) : m0, acc[2]);
            acc[3] = fma2(mul2(q0, m0), m1m1, fma2(mul2(q1, m1), m0m0, acc[3]));
        }
#pragma unroll
        for (int a = 0; a < 6; a++) {
            w[a][0] = w[a][1];
            w[a][1] = w[a][2];
        }
        fbz[0][0] = fbz[0][1];
        fbz[1][0] = fbz[1][1];
    };
    for (int k = 0; k < nz; k += 2) {
        plane_step(k, std::integral_constant<int, 0>{});
        if (k + 1 < nz) plane_step(k + 1, std::integral_constant<int, 1>{});
    }
    cp_async_wait(0);
    if (!sums) return;
    float v[kSums] = {lo2(acc[0]) + hi2(acc[0]), lo2(acc[1]) + hi2(acc[1]), lo2(acc[2]) + hi2(acc[2]),
                      lo2(acc[3]) + hi2(acc[3])};
    adj_finish(v, red, as, hist, partials, M);
}

// J = <f1^2> (volume mean of chi squared) per block, and its gradient 2 f1 / N^3.
template <typename T>
__global__ void __launch_bounds__(kAdjThreads) chi2_kernel(const T* __restrict__ f1, T* __restrict__ grad, long long n3,
                                                           double inv_sites, double* partials)
{
    __shared__ double red[32 * kSums];
    T acc[kSums] = {T(0), T(0), T(0), T(0)};
    const T two_over = (T)(2.0 * inv_sites);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (long long)gridDim.x * blockDim.x) {
        const T v = f1[i];
        acc[0] += v * v;
        if (grad) grad[i] = two_over * v;
    }
    double bs[kSums];
    block_reduce(acc, red, bs);
    if (threadIdx.x == 0) partials[blockIdx.x] = bs[0];
}

// Observable 1: the fraction of the energy density in chi at the momentum time
// of the final state, fields and a taken back half a step (f_t = f - (dt/2) pi,
// a_t = a - (dt/2) a', h = a'/a_t): K_i = <(pi_i - r h f_t,i)^2>/2,
// G_i = a_t^(-2s-2) <|grad+ f_t,i|^2>/2, W = <V_pr(f_t; a_t)>,
// J = (K_1 + G_1) / (K_0 + K_1 + G_0 + G_1 + W) (eq. rho-pres; the physical
// factor cancels in the ratio). FP64 arithmetic from the stored elements.
struct FracConst {
    double dt2, rh, cg, cd, kp, inv_dx2;
    int beta;
};
constexpr int kFracSums = 8;   // sum u0^2, u1^2, |d+ f_t0|^2, |d+ f_t1|^2, f_t0^beta/beta, f_t0^2 f_t1^2/2, u0 f_t0, u1 f_t1

template <typename T>
__device__ __forceinline__ double ft_at(const T* f, const T* p, size_t i, double dt2)
{
    return (double)f[i] - dt2 * (double)p[i];
}

template <typename T>
__global__ void __launch_bounds__(kAdjThreads) frac_sums_kernel(const T* __restrict__ f0, const T* __restrict__ f1,
                                                                const T* __restrict__ p0, const T* __restrict__ p1,
                                                                int n, FracConst c, double* partials)
{
    __shared__ double red[kAdjThreads / 32][kFracSums];
    double acc[kFracSums] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    const long long n3 = (long long)n * n * n;
    const T* f[2] = {f0, f1};
    const T* p[2] = {p0, p1};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % n), y = (int)((i / n) % n), z = (int)(i / ((long long)n * n));
        const size_t nb[3] = {((size_t)z * n + y) * n + (x == n - 1 ? 0 : x + 1),
                              ((size_t)z * n + (y == n - 1 ? 0 : y + 1)) * n + x,
                              ((size_t)(z == n - 1 ? 0 : z + 1) * n + y) * n + x};
        double t[2];
        for (int k = 0; k < 2; k++) {
            t[k] = ft_at(f[k], p[k], (size_t)i, c.dt2);
            const double u = (double)p[k][i] - c.rh * t[k];
            acc[k] += u * u;
            acc[6 + k] += u * t[k];
            double g = 0.0;
            for (int d = 0; d < 3; d++) {
                const double e = ft_at(f[k], p[k], nb[d], c.dt2) - t[k];
                g += e * e;
            }
            acc[2 + k] += g;
        }
        const double sq = t[0] * t[0];
        acc[4] += c.beta == 4 ? 0.25 * sq * sq : 0.5 * sq;
        acc[5] += 0.5 * sq * t[1] * t[1];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < kFracSums; k++) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < kFracSums) {
        double v = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) v += red[w][threadIdx.x];
        partials[(size_t)blockIdx.x * kFracSums + threadIdx.x] = v;
    }
}

// dJ/df and dJ/dpi of the stored final state: with dJ = (dN - J dD)/D, weights
// w_i on field i's own kinetic and gradient terms ((1 - J)/D for chi, -J/D for
// phi) and wW = -J/D on W,
//   g_i = (w_i (-r h u_i - a_t^(-2s-2) L f_t,i) + wW dV_pr/df_t,i) / N^3,
//   dJ/df_i = g_i, dJ/dpi_i = w_i u_i / N^3 - (dt/2) g_i  (u_i = pi_i - r h f_t,i).
template <typename T>
__global__ void __launch_bounds__(kAdjThreads) frac_seed_kernel(const T* __restrict__ f0, const T* __restrict__ f1,
                                                                const T* __restrict__ p0, const T* __restrict__ p1,
                                                                int n, FracConst c, double w0, double w1, double wW,
                                                                double inv_sites, T* __restrict__ fb, T* __restrict__ pb)
{
    const long long n3 = (long long)n * n * n;
    const T* f[2] = {f0, f1};
    const T* p[2] = {p0, p1};
    const double w[2] = {w0, w1};
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % n), y = (int)((i / n) % n), z = (int)(i / ((long long)n * n));
        const int xm = x == 0 ? n - 1 : x - 1, xp = x == n - 1 ? 0 : x + 1;
        const int ym = y == 0 ? n - 1 : y - 1, yp = y == n - 1 ? 0 : y + 1;
        const int zm = z == 0 ? n - 1 : z - 1, zp = z == n - 1 ? 0 : z + 1;
        const size_t nb[6] = {((size_t)z * n + y) * n + xm,  ((size_t)z * n + y) * n + xp,
                              ((size_t)z * n + ym) * n + x,  ((size_t)z * n + yp) * n + x,
                              ((size_t)zm * n + y) * n + x,  ((size_t)zp * n + y) * n + x};
        double t[2], lap[2];
        for (int k = 0; k < 2; k++) {
            t[k] = ft_at(f[k], p[k], (size_t)i, c.dt2);
            double l = 0.0;
            for (int d = 0; d < 6; d++) l += ft_at(f[k], p[k], nb[d], c.dt2) - t[k];
            lap[k] = l * c.inv_dx2;
        }
        const double dW[2] = {c.cd * (c.beta == 4 ? t[0] * t[0] * t[0] : t[0]) + c.kp * t[0] * t[1] * t[1],
                              c.kp * t[0] * t[0] * t[1]};
        for (int k = 0; k < 2; k++) {
            const double u = (double)p[k][i] - c.rh * t[k];
            const double g = (w[k] * (-c.rh * u - c.cg * lap[k]) + wW * dW[k]) * inv_sites;
            fb[(size_t)k * n3 + i] = (T)g;
            pb[(size_t)k * n3 + i] = (T)(w[k] * u * inv_sites - c.dt2 * g);
        }
    }
}

int adj_blocks(long long n3)
{
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long need = (n3 + kAdjThreads - 1) / kAdjThreads;
    return (int)std::max<long long>(1, std::min<long long>(need, (long long)sms * 8));
}

// z chunks per tile column of the reverse kernels: the launch runs in
// ceil(tiles * nzc / slots) waves of blocks that each march n / nzc planes and
// stage two halo planes more, so pick the nzc (at least 8 planes per chunk) that
// minimises waves x (planes per block + 2), the fewest chunks among equals.
// `slots` = resident blocks on the device.
int adj_zchunks(int n, int tiles, int slots)
{
    slots = std::max(1, slots);
    int best = 1;
    double best_t = 1e300;
    for (int nzc = 1; nzc <= std::max(1, n / 8); nzc++) {
        const long long waves = ((long long)tiles * nzc + slots - 1) / slots;
        const double t = (double)waves * ((n + nzc - 1) / nzc + 2);
        if (t < best_t - 1e-9) {
            best_t = t;
            best = nzc;
        }
    }
    return best;
}

int resident_slots(const void* fn, int threads, size_t smem)
{
    int dev = 0, sms = 148, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem) != cudaSuccess || occ < 1) occ = 1;
    return sms * occ;
}

// The history pointer of a scalar block (DevScalars::log, log_base).
struct LogField {
    DevScalars* log;
    long long log_base;
};
static_assert(offsetof(DevScalars, log_base) == offsetof(DevScalars, log) + sizeof(DevScalars*),
              "log and log_base are adjacent");

// Clears the history pointer of the handle's scalar block when armed: the
// pointer refers to scratch that the call frees, so no later step may see it.
// Declared after the call's Scratch, so it runs (and waits for the clear)
// before the scratch is freed.
struct LogGuard {
    DevScalars* sc;
    cudaStream_t st;
    bool armed = false;
    lat_status clear()
    {
        if (!armed) return LAT_OK;
        static const LogField zero{nullptr, 0};
        if (cudaMemcpyAsync((unsigned char*)sc + offsetof(DevScalars, log), &zero, sizeof(zero),
                            cudaMemcpyHostToDevice, st) != cudaSuccess)
            return LAT_ECUDA;
        armed = false;
        return LAT_OK;
    }
    ~LogGuard()
    {
        if (armed && clear() == LAT_OK) cudaStreamSynchronize(st);
    }
};

// Device allocations of one reverse-mode call, freed together.
struct Scratch {
    std::vector<void*> ptrs;
    ~Scratch()
    {
        for (void* p : ptrs) cudaFree(p);
    }
    template <typename P>
    bool alloc(P** out, size_t bytes)
    {
        void* p = nullptr;
        if (cudaMalloc(&p, std::max<size_t>(bytes, 16)) != cudaSuccess) return false;
        ptrs.push_back(p);
        *out = static_cast<P*>(p);
        return true;
    }
};

// Reverse-mode product of n steps. If observable >= 0 the adjoint of the final
// state is that of the observable (0: <chi^2>; 1: the fraction of the energy
// density in chi), written into fb/pb (and, for 1, into the adjoints of a, a'
// and kappa0) after the
// forward pass, and *J_out receives its value; otherwise fb, pb and sbar[0..1]
// carry the adjoint of the final state in.
template <typename T>
lat_status vjp_impl(lat_handle* h, int64_t n, int64_t ckpt_every, T* fb_user, T* pb_user, double sbar[4],
                    int observable, double* J_out)
{
    const Model& M = h->M;
    const size_t N3 = h->nsites, ab = N3 * sizeof(T);
    cudaStream_t st = h->stream;
    lat_status rs = ensure_prepared(h);
    if (rs != LAT_OK) return rs;
    DevScalars s0;
    rs = read_scalars(h, &s0);
    if (rs != LAT_OK) return rs;
    if (s0.status != LAT_OK) return (lat_status)s0.status;
    const int64_t K = ckpt_every > 0 ? std::min<int64_t>(ckpt_every, std::max<int64_t>(n, 1))
                                     : std::max<int64_t>(1, (int64_t)std::ceil(std::sqrt((double)n)));
    const int64_t nck = n > 0 ? (n + K - 1) / K : 0;
    const int nb = adj_blocks((long long)N3);
    // FP32 lattices with N a multiple of 64 take the two-site kernel, other
    // multiples of 32 the one-site z-march, the rest one site per thread
    bool pair = false;
    if constexpr (sizeof(T) == 4)
        pair = M.n % (2 * kPX) == 0 &&
               allow_dynamic_smem((const void*)adj_pair_kernel, sizeof(AdjPairSmem)) == cudaSuccess;
    const bool march = !pair && M.n % kMX == 0 &&
                       allow_dynamic_smem((const void*)adj_march_kernel<T>, adj_march_smem<T>()) == cudaSuccess;
    const int nzc =
        pair ? adj_zchunks(M.n, (M.n / (2 * kPX)) * (M.n / kPY),
                           resident_slots((const void*)adj_pair_kernel, kPX * kPY, sizeof(AdjPairSmem)))
        : march ? adj_zchunks(M.n, (M.n / kMX) * (M.n / kMY),
                              resident_slots((const void*)adj_march_kernel<T>, kMX * kMY, adj_march_smem<T>()))
                : 0;
    const dim3 mgrid(pair ? M.n / (2 * kPX) : march ? M.n / kMX : 1, pair ? M.n / kPY : march ? M.n / kMY : 1,
                     (pair || march) ? nzc : 1);
    const size_t nparts = std::max<size_t>(nb, (size_t)mgrid.x * mgrid.y * mgrid.z);

    Scratch S;
    T *ck = nullptr, *seg = nullptr, *adj1 = nullptr, *fin = nullptr;
    DevScalars *ck_sc = nullptr, *hist = nullptr, *fin_sc = nullptr;
    AdjScalars* as = nullptr;
    double* part = nullptr;
    if (!S.alloc(&ck, (size_t)nck * 6 * ab) || !S.alloc(&ck_sc, (size_t)nck * sizeof(DevScalars)) ||
        !S.alloc(&hist, (size_t)(n + 1) * sizeof(DevScalars)) || !S.alloc(&seg, (size_t)K * 2 * ab) ||
        !S.alloc(&adj1, 4 * ab) || !S.alloc(&fin, 4 * ab) || !S.alloc(&fin_sc, sizeof(DevScalars)) ||
        !S.alloc(&as, sizeof(AdjScalars)) ||
        !S.alloc(&part, std::max(nparts * kSums, (size_t)nb * kFracSums) * sizeof(double)))
        return LAT_ENOMEM;
    Bufs<T> hb = bufs_of<T>(h);
    auto arr = [&](T* base, size_t i) { return base + i * N3; };

    // forward pass: checkpoints (f_c, pi_c, f_{c-1}, scalars) every K steps and
    // the scalars every step started from: hist[0] copied here, hist[k + 1]
    // stored by step k's last block while the handle's scalar block carries the
    // history pointer (cleared below, and by the guard on every early return)
    LogGuard guard{h->sc, st};
    {
        const LogField lf{hist, (long long)s0.step};
        LAT_CUDA(cudaMemcpyAsync((unsigned char*)h->sc + offsetof(DevScalars, log), &lf, sizeof(lf),
                                 cudaMemcpyHostToDevice, st));
        guard.armed = true;
    }
    LAT_CUDA(cudaMemcpyAsync(hist, h->sc, sizeof(DevScalars), cudaMemcpyDeviceToDevice, st));
    for (int64_t k = 0; k < n; k++) {
        const int par = (int)((s0.step + k) & 1);
        if (k % K == 0) {
            T* c = arr(ck, (size_t)(k / K) * 6);
            for (int f = 0; f < 2; f++) {
                LAT_CUDA(cudaMemcpyAsync(c + f * N3, hb.f[par][f], ab, cudaMemcpyDeviceToDevice, st));
                LAT_CUDA(cudaMemcpyAsync(c + (2 + f) * N3, hb.p[par][f], ab, cudaMemcpyDeviceToDevice, st));
                if (k > 0) LAT_CUDA(cudaMemcpyAsync(c + (4 + f) * N3, hb.f[1 - par][f], ab, cudaMemcpyDeviceToDevice, st));
            }
            LAT_CUDA(cudaMemcpyAsync(ck_sc + k / K, h->sc, sizeof(DevScalars), cudaMemcpyDeviceToDevice, st));
        }
        LAT_CUDA(launch_step_with<T>(h, hb, false));
    }
    LAT_TRY(guard.clear());
    const int parN = (int)((s0.step + n) & 1);
    for (int f = 0; f < 2; f++) {
        LAT_CUDA(cudaMemcpyAsync(fin + f * N3, hb.f[parN][f], ab, cudaMemcpyDeviceToDevice, st));
        LAT_CUDA(cudaMemcpyAsync(fin + (2 + f) * N3, hb.p[parN][f], ab, cudaMemcpyDeviceToDevice, st));
    }
    LAT_CUDA(cudaMemcpyAsync(fin_sc, h->sc, sizeof(DevScalars), cudaMemcpyDeviceToDevice, st));

    // adjoint of the final state
    AdjScalars a0;
    std::memset(&a0, 0, sizeof(a0));
    if (observable == 0) {
        LAT_CUDA(cudaMemsetAsync(fb_user, 0, ab, st));
        LAT_CUDA(cudaMemsetAsync(pb_user, 0, 2 * ab, st));
        chi2_kernel<T><<<nb, kAdjThreads, 0, st>>>(hb.f[parN][1], fb_user + N3, (long long)N3, M.inv_sites, part);
        LAT_CUDA(cudaGetLastError());
        std::vector<double> hp(nb);
        LAT_CUDA(cudaMemcpyAsync(hp.data(), part, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
        LAT_CUDA(cudaStreamSynchronize(st));
        double J = 0.0;
        for (int b = 0; b < nb; b++) J += hp[b];
        if (J_out) *J_out = J * M.inv_sites;
    } else if (observable == 1) {
        DevScalars sF;
        LAT_CUDA(cudaMemcpyAsync(&sF, fin_sc, sizeof(sF), cudaMemcpyDeviceToHost, st));
        LAT_CUDA(cudaStreamSynchronize(st));
        const double at = sF.a - 0.5 * M.dt * sF.ad;
        const double h = M.expansion ? sF.ad / at : 0.0;
        FracConst c;
        c.dt2 = 0.5 * M.dt;
        c.rh = M.r * h;
        c.cg = std::pow(at, -2.0 * M.s - 2.0);
        c.cd = M.cdom0 * std::pow(at, M.pdom);
        c.kp = M.kappa0 * std::pow(at, M.pint);
        c.inv_dx2 = M.inv_dx2;
        c.beta = M.beta;
        const T *F0 = hb.f[parN][0], *F1 = hb.f[parN][1], *P0 = hb.p[parN][0], *P1 = hb.p[parN][1];
        frac_sums_kernel<T><<<nb, kAdjThreads, 0, st>>>(F0, F1, P0, P1, M.n, c, part);
        LAT_CUDA(cudaGetLastError());
        std::vector<double> hp((size_t)nb * kFracSums);
        LAT_CUDA(cudaMemcpyAsync(hp.data(), part, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        LAT_CUDA(cudaStreamSynchronize(st));
        double S[kFracSums] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        for (int b = 0; b < nb; b++)
            for (int k = 0; k < kFracSums; k++) S[k] += hp[(size_t)b * kFracSums + k];
        const double is = M.inv_sites;
        const double K0 = 0.5 * S[0] * is, K1 = 0.5 * S[1] * is;
        const double G0 = 0.5 * c.cg * S[2] * M.inv_dx2 * is, G1 = 0.5 * c.cg * S[3] * M.inv_dx2 * is;
        const double Wd = S[4] * is, Wi = S[5] * is, UF0 = S[6] * is, UF1 = S[7] * is;
        const double W = c.cd * Wd + c.kp * Wi, D = K0 + K1 + G0 + G1 + W, J = (K1 + G1) / D;
        if (!std::isfinite(J) || !(D != 0.0)) return LAT_ENONFINITE;
        if (J_out) *J_out = J;
        const double w0 = -J / D, w1 = (1.0 - J) / D, wW = -J / D;
        frac_seed_kernel<T><<<nb, kAdjThreads, 0, st>>>(F0, F1, P0, P1, M.n, c, w0, w1, wW, is, fb_user, pb_user);
        LAT_CUDA(cudaGetLastError());
        const double dJ_dh = w0 * (-M.r * UF0) + w1 * (-M.r * UF1);
        const double dJ_dat = (w0 * G0 + w1 * G1) * (-2.0 * M.s - 2.0) / at + wW * (M.pdom * c.cd * Wd + M.pint * c.kp * Wi) / at;
        if (M.expansion) {
            a0.ba = dJ_dat + dJ_dh * (-sF.ad / (at * at));
            a0.bad = -0.5 * M.dt * dJ_dat + dJ_dh * (1.0 / at + 0.5 * M.dt * sF.ad / (at * at));
        }
        a0.bk0 = wW * Wi * std::pow(at, M.pint);   // J's own dependence on kappa0 (the interaction energy)
    } else {
        a0.ba = sbar[0];
        a0.bad = sbar[1];
    }
    LAT_CUDA(cudaMemcpyAsync(as, &a0, sizeof(a0), cudaMemcpyHostToDevice, st));

    T* setF[2] = {fb_user, adj1};
    T* setP[2] = {pb_user, adj1 + 2 * N3};
    int cur = 0;
    auto adj_bufs = [&](const T* fk0, const T* fm0) {
        AdjBufs<T> b;
        for (int f = 0; f < 2; f++) {
            b.f[f] = fk0 ? fk0 + f * N3 : nullptr;
            b.fm[f] = fm0 ? fm0 + f * N3 : nullptr;
            b.fb[f] = setF[cur] + f * N3;
            b.pb[f] = setP[cur] + f * N3;
            b.fbo[f] = setF[1 - cur] + f * N3;
            b.pbo[f] = setP[1 - cur] + f * N3;
        }
        return b;
    };
    if (n > 0) {
        // sums of the last step from the final adjoint and f_{n-1}, still in
        // the other ping-pong buffer
        T* fm_last = seg;   // f_{n-1} copied next to the segment storage
        for (int f = 0; f < 2; f++)
            LAT_CUDA(cudaMemcpyAsync(fm_last + f * N3, hb.f[1 - parN][f], ab, cudaMemcpyDeviceToDevice, st));
        adj_step_kernel<T, false><<<nb, kAdjThreads, 0, st>>>(adj_bufs(nullptr, fm_last), M, as, hist + (n - 1), part);
        LAT_CUDA(cudaGetLastError());
    }
    for (int64_t sgi = nck - 1; sgi >= 0; sgi--) {
        const int64_t c = sgi * K, e = std::min<int64_t>(c + K, n);
        const T* cp = arr(ck, (size_t)sgi * 6);
        // restore the checkpoint and recompute f_c .. f_{e-1} into the segment storage
        const int parc = (int)((s0.step + c) & 1);
        for (int f = 0; f < 2; f++) {
            LAT_CUDA(cudaMemcpyAsync(seg + f * N3, cp + f * N3, ab, cudaMemcpyDeviceToDevice, st));
            LAT_CUDA(cudaMemcpyAsync(hb.p[parc][f], cp + (2 + f) * N3, ab, cudaMemcpyDeviceToDevice, st));
        }
        LAT_CUDA(cudaMemcpyAsync(h->sc, ck_sc + sgi, sizeof(DevScalars), cudaMemcpyDeviceToDevice, st));
        guard.armed = true;   // the checkpoint's block carries the history pointer
        LAT_TRY(guard.clear());
        for (int64_t k = c; k + 1 < e; k++) {
            const int par = (int)((s0.step + k) & 1);
            Bufs<T> b = hb;
            for (int f = 0; f < 2; f++) {
                b.f[par][f] = arr(seg, (size_t)(k - c) * 2 + f);
                b.f[1 - par][f] = arr(seg, (size_t)(k - c + 1) * 2 + f);
            }
            LAT_CUDA(launch_step_with<T>(h, b, false));
        }
        // reverse steps e-1 .. c
        for (int64_t k = e - 1; k >= c; k--) {
            const T* fk = arr(seg, (size_t)(k - c) * 2);
            const T* fm = k > c ? arr(seg, (size_t)(k - c - 1) * 2) : (k > 0 ? cp + 4 * N3 : nullptr);
            if constexpr (sizeof(T) == 4) {
                if (pair) {
                    adj_pair_kernel<<<mgrid, dim3(kPX, kPY), sizeof(AdjPairSmem), st>>>(
                        adj_bufs(fk, fm), M, as, k > 0 ? hist + (k - 1) : hist, part, nzc);
                    LAT_CUDA(cudaGetLastError());
                    cur = 1 - cur;
                    continue;
                }
            }
            if (march)
                adj_march_kernel<T><<<mgrid, dim3(kMX, kMY), adj_march_smem<T>(), st>>>(
                    adj_bufs(fk, fm), M, as, k > 0 ? hist + (k - 1) : hist, part, nzc);
            else
                adj_step_kernel<T, true><<<nb, kAdjThreads, 0, st>>>(adj_bufs(fk, fm), M, as,
                                                                     k > 0 ? hist + (k - 1) : hist, part);
            LAT_CUDA(cudaGetLastError());
            cur = 1 - cur;
        }
    }
    if (cur != 0) {
        LAT_CUDA(cudaMemcpyAsync(fb_user, setF[cur], 2 * ab, cudaMemcpyDeviceToDevice, st));
        LAT_CUDA(cudaMemcpyAsync(pb_user, setP[cur], 2 * ab, cudaMemcpyDeviceToDevice, st));
    }
    // the handle ends at the final state
    for (int f = 0; f < 2; f++) {
        LAT_CUDA(cudaMemcpyAsync(hb.f[parN][f], fin + f * N3, ab, cudaMemcpyDeviceToDevice, st));
        LAT_CUDA(cudaMemcpyAsync(hb.p[parN][f], fin + (2 + f) * N3, ab, cudaMemcpyDeviceToDevice, st));
    }
    LAT_CUDA(cudaMemcpyAsync(h->sc, fin_sc, sizeof(DevScalars), cudaMemcpyDeviceToDevice, st));
    AdjScalars out;
    LAT_CUDA(cudaMemcpyAsync(&out, as, sizeof(out), cudaMemcpyDeviceToHost, st));
    DevScalars sN;
    LAT_CUDA(cudaMemcpyAsync(&sN, fin_sc, sizeof(sN), cudaMemcpyDeviceToHost, st));
    LAT_CUDA(cudaStreamSynchronize(st));
    if (sN.status != LAT_OK) return (lat_status)sN.status;
    if (out.status != LAT_OK) return (lat_status)out.status;
    sbar[0] = out.ba;
    sbar[1] = out.bad;
    sbar[2] = out.bk0;
    sbar[3] = out.bk0 / (M.A * M.A * M.B * M.B);
    return LAT_OK;
}

} // namespace

} // namespace lat

using namespace lat;

extern "C" {

lat_status lat_vjp(lat_handle* h, int64_t n_steps, int64_t ckpt_every, void* fbar_dev, void* pibar_dev,
                   double sbar[4])
{
    if (!h || n_steps < 0 || ckpt_every < 0 || !fbar_dev || !pibar_dev || !sbar) return LAT_EINVAL;
    if (h->slab) return LAT_ESTATE;
    if (h->M.stencil == 27) return LAT_EUNSUPPORTED;   // the reverse step is written for 7 points
    if (h->M.expansion == 2) return LAT_EUNSUPPORTED;  // and for eq. scale
    if (h->M.split) return LAT_EUNSUPPORTED;           // and for phi stored whole
    if (((uintptr_t)fbar_dev | (uintptr_t)pibar_dev) % h->esize != 0) return LAT_EINVAL;
    return h->prec == 32 ? vjp_impl<float>(h, n_steps, ckpt_every, (float*)fbar_dev, (float*)pibar_dev, sbar, -1, nullptr)
                         : vjp_impl<double>(h, n_steps, ckpt_every, (double*)fbar_dev, (double*)pibar_dev, sbar, -1,
                                            nullptr);
}

lat_status lat_adjoint(lat_handle* h, int64_t n_steps, int observable, int64_t ckpt_every, double* J_out,
                       double* dJ_dg2, void* dJ_df_dev, void* dJ_dpi_dev)
{
    if (!h || n_steps < 0 || ckpt_every < 0 || !dJ_df_dev || !dJ_dpi_dev) return LAT_EINVAL;
    if (h->slab) return LAT_ESTATE;
    if (h->M.stencil == 27 || h->M.expansion == 2 || h->M.split) return LAT_EUNSUPPORTED;
    if (observable != 0 && observable != 1) return LAT_EUNSUPPORTED;
    if (((uintptr_t)dJ_df_dev | (uintptr_t)dJ_dpi_dev) % h->esize != 0) return LAT_EINVAL;
    double sbar[4] = {0.0, 0.0, 0.0, 0.0};
    const lat_status st =
        h->prec == 32 ? vjp_impl<float>(h, n_steps, ckpt_every, (float*)dJ_df_dev, (float*)dJ_dpi_dev, sbar, observable, J_out)
                      : vjp_impl<double>(h, n_steps, ckpt_every, (double*)dJ_df_dev, (double*)dJ_dpi_dev, sbar, observable,
                                         J_out);
    if (st == LAT_OK && dJ_dg2) *dJ_dg2 = sbar[3];
    return st;
}

} // extern "C"
