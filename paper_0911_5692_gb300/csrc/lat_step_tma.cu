// lat_step_tma.cu -- the fused leapfrog step on sm_103a with a TMA plane ring.
//
// The step is that of lat_step_simple.cu (Sec. II.B, eq. evo with eq.
// scalar-evo: 7-point Laplacian, potential derivative, kick and drift of both
// fields; the sums of the new fields for eq. scale from a one-site look-ahead
// rim; the FP64 a(t) update in the last block), laid out for the GB300 memory
// system:
//
// * A block owns full x rows (x wraps inside shared memory), `ty` rows in y and a
//   chunk of `zr` planes in z, and marches the chunk in +z. The paper's Fig. 1
//   marches whole z columns through three shared-memory planes; here each
//   z-plane of the tile (with a 1-row halo below and a 2-row halo above, the
//   second one for the look-ahead rim) is one ring slot filled by the Tensor
//   Memory Accelerator: 1-row boxes `cp.async.bulk.tensor.3d` with periodic
//   y and z coordinates computed on the fly, completion tracked by an mbarrier
//   per slot. `depth` planes are in flight ahead of the plane being computed.
// * Threads own 16-byte vectors of a row (4 floats or 2 doubles): every global
//   store is a coalesced 16-byte store and the stencil reads are 16-byte shared
//   loads plus two scalar loads for the x neighbours.
// * The new fields go to shared memory once more so the forward differences
//   in x and y (including the look-ahead row) can be summed; the z difference
//   uses the previous plane kept in registers. Sums accumulate in FP32 per
//   thread, FP64 per block.
// * Every wait is bounded (%globaltimer); a block that times out raises
//   LAT_ETIMEOUT, skips its global writes, keeps every barrier and waits
//   (bounded) for its own copies in flight before it exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>

#include "lat_kernels.h"
#include "lat_pairs.cuh"

namespace lat {

namespace {

constexpr unsigned long long kWaitNs = 1000ull * 1000ull * 1000ull;   // 1 s per wait
constexpr int kMaxThreads = 768;   // up to 85 registers per thread


template <typename T>
struct TmaArgs {
    CUtensorMap maps[kTmaMaps];   // one-row boxes of f0, f1, p0, p1 (set 0, then set 1), then tall boxes
    Bufs<T> b;
    Model M;
    DevScalars* sc;
    double* partials;
    TmaGeom g;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the completion of phase `parity` of an mbarrier. On timeout
// the block's abort flag is raised and the wait gives up.
__device__ __forceinline__ void mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort)
{
    if (*abort) return;
    if (mbar_try_wait(bar, parity)) return;
    const unsigned long long t0 = gtimer();
    while (!mbar_try_wait(bar, parity)) {
        if (gtimer() - t0 > kWaitNs) {
            *abort = 1;
            return;
        }
    }
}

__device__ __forceinline__ void tma_load_row(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(dst),
        "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Issue the TMA loads of one f plane (both fields, rows y0-1 .. y0+ty+1) or one
// momentum plane (both fields, rows y0 .. y0+ty) into a ring slot; warp 0 only.
// Shared layout of a slot: [field][x chunk][row][bw], row stride G.rs. Where the
// rows do not wrap around the periodic y boundary, one multi-row box per field
// and x chunk; otherwise one box per row with the wrapped y coordinate.
template <typename T>
__device__ __forceinline__ void issue_plane(const TmaArgs<T>& A, int par, bool momentum, unsigned char* slot,
                                            uint32_t bar, int y0, int z)
{
    const TmaGeom& G = A.g;
    const int lane = threadIdx.x & 31;
    const int rows = momentum ? G.ty + 1 : G.ty + 3;
    const int ylo = momentum ? y0 : y0 - 1;
    const uint32_t cs = (uint32_t)rows * G.rs, fsz = cs * G.nbx;
    const int mi = 4 * par + (momentum ? 2 : 0);
    if (lane == 0) mbar_expect_tx(bar, (uint32_t)(2 * rows * G.n * (int)sizeof(T)));
    __syncwarp();
    if (G.tall && ylo >= 0 && ylo + rows <= G.n) {
        for (int i = lane; i < 2 * G.nbx; i += 32) {
            const int field = i / G.nbx, bx = i - field * G.nbx;
            tma_load_row(smem_u32(slot + field * fsz + bx * cs), &A.maps[8 + mi + field], bx * G.bw, ylo, z, bar);
        }
    } else {
        const int boxes = 2 * rows * G.nbx;
        for (int i = lane; i < boxes; i += 32) {
            const int field = i / (rows * G.nbx);
            const int rem = i - field * rows * G.nbx;
            const int bx = rem / rows, r = rem - bx * rows;
            tma_load_row(smem_u32(slot + field * fsz + bx * cs + r * G.rs), &A.maps[mi + field], bx * G.bw,
                         wrapi(ylo + r, G.n), z, bar);
        }
    }
}

// Per-thread item: one 16-byte vector (NP pairs) of one field in row r of the
// tile. Items are ordered field, row, x so that the lanes of a warp hold
// consecutive vectors of a row and exchange x neighbours by shuffles.
struct ItemOff {
    uint32_t c;    // centre of this field, f slot
    uint32_t xl;   // left neighbour of the first site, f slot
    uint32_t xr;   // right neighbour of the last site, f slot
    uint32_t p;    // this field's momenta / new-field buffer
    uint32_t pxr;  // new-field buffer, right neighbour
    uint32_t rx;   // r * n + x: offset of the vector inside its tile plane
    int r;         // row in the tile, -1 for an idle thread
    int flags;     // bit 0: field 1; bit 1: left neighbour in lane - 1; bit 2: right in lane + 1
};

template <typename T>
__device__ __forceinline__ T shfl_up1(T v) { return __shfl_up_sync(0xffffffffu, v, 1); }
template <typename T>
__device__ __forceinline__ T shfl_down1(T v) { return __shfl_down_sync(0xffffffffu, v, 1); }

template <typename T, int IPT>
__global__ void __launch_bounds__(kMaxThreads) step_tma_kernel(const __grid_constant__ TmaArgs<T> A)
{
    typedef typename PK<T>::P P;
    constexpr int NP = PK<T>::NP;
    constexpr int VW = 2 * NP;
    constexpr uint32_t E = sizeof(T);
    const TmaGeom& G = A.g;
    const Model& M = A.M;
    DevScalars* sc = A.sc;
    if (sc->status != LAT_OK) return;

    extern __shared__ unsigned char smem_raw[];
    // 128-byte aligned start, kept as an offset into the shared array so every
    // access stays a shared-memory access
    unsigned char* base = smem_raw + ((128u - (smem_u32(smem_raw) & 127u)) & 127u);
    const uint32_t rowB = (uint32_t)G.rs;
    const uint32_t fieldF = (uint32_t)(G.ty + 3) * rowB * G.nbx, fieldP = (uint32_t)(G.ty + 1) * rowB * G.nbx;
    const uint32_t fslotB = 2u * fieldF, pslotB = 2u * fieldP;
    unsigned char* fs = base;
    unsigned char* ps = fs + G.rf * fslotB;
    unsigned char* gbuf = ps + G.rp * pslotB;                  // two buffers of new fields
    uint64_t* bars = (uint64_t*)(gbuf + 2 * pslotB);            // rf + rp mbarriers
    double* red = (double*)(bars + G.rf + G.rp + 1);
    __shared__ int abort_flag;
    volatile int* abort = &abort_flag;

    const int n = G.n;
    const int par = (int)(sc->step & 1);
    // f' += dt (cL Lap f + cF f - dV/df), f += dt f': coefficients folded so that
    // the unscaled neighbour-difference sum multiplies dt cL / dx^2 directly
    const T dt_s = step_coef<T>(sc, 4);
    const T dtcl = step_coef<T>(sc, 0), dtcf = step_coef<T>(sc, 1);
    const T mdtcdom = step_coef<T>(sc, 2), mdtkap = step_coef<T>(sc, 3);
    const bool quartic = M.beta == 4;

    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < G.rf + G.rp; s++) mbar_init(smem_u32(&bars[s]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int Q = n / VW;

    // byte offset of site (row, x) inside one field block: [x chunk][row][bw]
    auto offs = [&](int rows, int row, int x) -> uint32_t {
        const int bx = x / G.bw;
        return ((uint32_t)bx * rows + row) * rowB + (uint32_t)(x - bx * G.bw) * E;
    };
    ItemOff io[IPT];
#pragma unroll
    for (int it = 0; it < IPT; it++) {
        const int item = threadIdx.x + it * blockDim.x;
        const int valid = item < G.items;
        const int ii = valid ? item : 0;
        const int f = ii / ((G.ty + 1) * Q);
        const int rem = ii - f * (G.ty + 1) * Q;
        const int r = rem / Q, q = rem - r * Q, x = q * VW;
        const int xl = x == 0 ? n - 1 : x - 1, xr = x + VW == n ? 0 : x + VW;
        io[it].r = valid ? r : -1;
        io[it].rx = (uint32_t)r * n + x;
        io[it].c = f * fieldF + offs(G.ty + 3, r + 1, x);
        io[it].xl = f * fieldF + offs(G.ty + 3, r + 1, xl);
        io[it].xr = f * fieldF + offs(G.ty + 3, r + 1, xr);
        io[it].p = f * fieldP + offs(G.ty + 1, r, x);
        io[it].pxr = f * fieldP + offs(G.ty + 1, r, xr);
        io[it].flags = f | ((q > 0 && lane > 0) ? 2 : 0) | ((q < Q - 1 && lane < 31) ? 4 : 0);
    }

    // This block's share of the (y tile, z plane) index space: a contiguous run,
    // split at y-tile boundaries into segments marched in +z.
    const long long total = (long long)G.nyt * n;
    long long s0 = (long long)blockIdx.x * total / gridDim.x;
    const long long s1 = (long long)(blockIdx.x + 1) * total / gridDim.x;
    unsigned int fbase = 0, pbase = 0;     // f / momentum planes issued before this segment
    unsigned int f_issued = 0, p_issued = 0;

    // sums: |forward differences|^2 of the new field; f0^4 (or f0^2) and f0^2 f1^2
    P accg = mk2(T(0), T(0)), accvd = mk2(T(0), T(0)), accvi = mk2(T(0), T(0));
    const P dtcl2 = mk2(dtcl, dtcl), dtcf2 = mk2(dtcf, dtcf), dt2 = mk2(dt_s, dt_s);
    const P mdtcdom2 = mk2(mdtcdom, mdtcdom), mdtkap2 = mk2(mdtkap, mdtkap);

    while (s0 < s1) {
        const int yt = (int)(s0 / n), z0 = (int)(s0 - (long long)yt * n);
        const long long seg_end = min(s1, (long long)(yt + 1) * n);
        const int nz = (int)(seg_end - s0);
        const int y0 = yt * G.ty;
        const int nf = nz + 3, np_ = nz + 1;
        if (warp == 0 && !__shfl_sync(0xffffffffu, *abort, 0)) {
            for (int j = 0; j < min(nf, G.depth + 3); j++) {
                const unsigned int gj = fbase + j;
                issue_plane(A, par, false, fs + (gj % G.rf) * fslotB, smem_u32(&bars[gj % G.rf]), y0,
                            wrapi(z0 - 1 + j, n));
            }
            for (int k = 0; k < min(np_, G.depth + 1); k++) {
                const unsigned int gk = pbase + k;
                issue_plane(A, par, true, ps + (gk % G.rp) * pslotB, smem_u32(&bars[G.rf + gk % G.rp]), y0,
                            wrapi(z0 + k, n));
            }
            f_issued = fbase + min(nf, G.depth + 3);
            p_issued = pbase + min(np_, G.depth + 1);
        }

        for (int k = 0; k <= nz; k++) {
            if (k > 0 && warp == 0 && !__shfl_sync(0xffffffffu, *abort, 0)) {
                const int j = k + 2 + G.depth;
                if (j < nf) {
                    const unsigned int gj = fbase + j;
                    issue_plane(A, par, false, fs + (gj % G.rf) * fslotB, smem_u32(&bars[gj % G.rf]), y0,
                                wrapi(z0 - 1 + j, n));
                    f_issued = gj + 1;
                }
                const int kp = k + G.depth;
                if (kp < np_) {
                    const unsigned int gk = pbase + kp;
                    issue_plane(A, par, true, ps + (gk % G.rp) * pslotB, smem_u32(&bars[G.rf + gk % G.rp]), y0,
                                wrapi(z0 + kp, n));
                    p_issued = gk + 1;
                }
            }
            // f planes k (z-1), k+1 (z) and k+2 (z+1), momenta of plane k
            for (int j = k; j < k + 3; j++)
                mbar_wait(smem_u32(&bars[(fbase + j) % G.rf]), ((fbase + j) / G.rf) & 1, abort);
            mbar_wait(smem_u32(&bars[G.rf + (pbase + k) % G.rp]), ((pbase + k) / G.rp) & 1, abort);
            const bool ahead = k == nz;
            const size_t zoff = ((size_t)(z0 + k) * n + y0) * n;  // tile origin in the plane (unused on the look-ahead plane)
            const unsigned char* Fm = fs + ((fbase + k) % G.rf) * fslotB;
            const unsigned char* Fc = fs + ((fbase + k + 1) % G.rf) * fslotB;
            const unsigned char* Fp = fs + ((fbase + k + 2) % G.rf) * fslotB;
            const unsigned char* Pc = ps + ((pbase + k) % G.rp) * pslotB;
            unsigned char* gw = gbuf + (k & 1) * pslotB;              // new fields of plane k
            const unsigned char* gr = gbuf + ((k + 1) & 1) * pslotB;  // new fields of plane k-1
            const bool write = !ahead && !*abort;

#pragma unroll
            for (int it = 0; it < IPT; it++) {
                const int r = io[it].r;
                const int f = io[it].flags & 1;
                // centre of this field; x neighbours from the adjacent lanes (every
                // lane takes part in the shuffles) or from shared memory at the
                // ends of a row and of a warp
                P a[NP];
                PK<T>::ld(Fc + io[it].c, a);
                T left = shfl_up1(hi2(a[NP - 1]));
                T right = shfl_down1(lo2(a[0]));
                if (!(io[it].flags & 2)) left = *(const T*)(Fc + io[it].xl);
                if (!(io[it].flags & 4)) right = *(const T*)(Fc + io[it].xr);
                P g[NP];
                const bool active = r >= 0 && !(ahead && r == G.ty);
                if (active) {
                    P up[NP], dn[NP], zm[NP], zp[NP], ot[NP], pv[NP];
                    PK<T>::ld(Fc + io[it].c - rowB, up);
                    PK<T>::ld(Fc + io[it].c + rowB, dn);
                    PK<T>::ld(Fm + io[it].c, zm);
                    PK<T>::ld(Fp + io[it].c, zp);
                    PK<T>::ld(Fc + (f ? io[it].c - fieldF : io[it].c + fieldF), ot);
                    PK<T>::ld(Pc + io[it].p, pv);
                    // x neighbours as pairs: (left, a0), (a1, a2), ... and (.., aN, right)
                    P lft[NP], rgt[NP];
                    if constexpr (NP == 2) {
                        T c0, c1, c2, c3;
                        un2(a[0], c0, c1);
                        un2(a[1], c2, c3);
                        lft[0] = mk2(left, c0);
                        lft[1] = mk2(c1, c2);
                        rgt[0] = lft[1];
                        rgt[1] = mk2(c3, right);
                    } else {
                        lft[0] = mk2(left, lo2(a[0]));
                        rgt[0] = mk2(hi2(a[0]), right);
                    }
                    P pn[NP];
#pragma unroll
                    for (int q = 0; q < NP; q++) {
                        const P c = a[q];
                        // Laplacian as a sum of neighbour differences: exact
                        // differences for f = const + small (Sterbenz)
                        const P lapu = add2(add2(add2(sub2(lft[q], c), sub2(rgt[q], c)),
                                                 add2(sub2(up[q], c), sub2(dn[q], c))),
                                            add2(sub2(zm[q], c), sub2(zp[q], c)));
                        P acc = fma2(dtcl2, lapu, fma2(dtcf2, c, pv[q]));
                        // potential: f0 gets -dt (cdom f0^(beta-1) + kappa f0 f1^2),
                        // f1 gets -dt kappa f0^2 f1
                        const P f0 = f == 0 ? c : ot[q], f1 = f == 0 ? ot[q] : c;
                        const P f0f1 = mul2(f0, f1);
                        if (f == 0) {
                            const P dom = quartic ? mul2(mul2(f0, f0), f0) : f0;
                            acc = fma2(mdtcdom2, dom, fma2(mdtkap2, mul2(f0f1, f1), acc));
                        } else {
                            acc = fma2(mdtkap2, mul2(f0f1, f0), acc);
                        }
                        pn[q] = acc;
                        g[q] = fma2(dt2, acc, c);
                    }
                    if (write && r < G.ty) {
                        const size_t gi = zoff + io[it].rx;
                        T* outp = f == 0 ? A.b.p[par ^ 1][0] : A.b.p[par ^ 1][1];
                        T* outf = f == 0 ? A.b.f[par ^ 1][0] : A.b.f[par ^ 1][1];
                        PK<T>::st(outp + gi, pn);
                        PK<T>::st(outf + gi, g);
                    }
                    if (!ahead) PK<T>::st(gw + io[it].p, g);
                }
                // sums over the owned rows: z pair (k-1, k), and the x and y pairs
                // and the potential of plane k-1 from the buffer written one plane ago
                if (k > 0) {
                    P gp[NP];
                    PK<T>::ld(gr + io[it].p, gp);
                    T xnext = shfl_down1(lo2(gp[0]));
                    if (!(io[it].flags & 4)) xnext = *(const T*)(gr + io[it].pxr);
                    if (r >= 0 && r < G.ty) {
                        P yn[NP], xn[NP];
                        PK<T>::ld(gr + io[it].p + rowB, yn);
                        if constexpr (NP == 2) {
                            T a0, a1, a2, a3;
                            un2(gp[0], a0, a1);
                            un2(gp[1], a2, a3);
                            xn[0] = mk2(a1, a2);
                            xn[1] = mk2(a3, xnext);
                        } else {
                            xn[0] = mk2(hi2(gp[0]), xnext);
                        }
#pragma unroll
                        for (int q = 0; q < NP; q++) {
                            const P dxv = sub2(xn[q], gp[q]), dyv = sub2(yn[q], gp[q]), dzv = sub2(g[q], gp[q]);
                            accg = fma2(dxv, dxv, fma2(dyv, dyv, fma2(dzv, dzv, accg)));
                        }
                        if (f == 0) {
                            P g1[NP];
                            PK<T>::ld(gr + io[it].p + fieldP, g1);
#pragma unroll
                            for (int q = 0; q < NP; q++) {
                                const P sq = mul2(gp[q], gp[q]);
                                accvd = quartic ? fma2(sq, sq, accvd) : add2(sq, accvd);
                                accvi = fma2(sq, mul2(g1[q], g1[q]), accvi);
                            }
                        }
                    }
                }
            }
            __syncthreads();
        }
        fbase += nf;
        pbase += np_;
        s0 = seg_end;
    }

    if (*abort) {
        // raise the error, then wait (bounded) for this block's copies in flight:
        // the last load issued into each slot completes after all earlier ones
        if (threadIdx.x == 0) {
            atomicCAS(&sc->status, (int)LAT_OK, (int)LAT_ETIMEOUT);
            for (int s = 0; s < G.rf + G.rp; s++) {
                const bool isf = s < G.rf;
                const unsigned int cnt = isf ? f_issued : p_issued, nslot = isf ? G.rf : G.rp;
                const unsigned int slot = isf ? s : s - G.rf;
                if (cnt <= slot) continue;
                const unsigned int last = slot + ((cnt - 1 - slot) / nslot) * nslot;
                const unsigned long long t0 = gtimer();
                while (!mbar_try_wait(smem_u32(&bars[s]), (last / nslot) & 1) && gtimer() - t0 < kWaitNs) {}
            }
        }
        __syncthreads();
    }
    // per-thread sums to the block: gradient sums go to the thread's field,
    // the potential sums (with their 1/beta and 1/2 factors) come from field 0
    const T gsum = lo2(accg) + hi2(accg);
    const bool f0t = (io[0].flags & 1) == 0;
    T v[kSums] = {f0t ? gsum : T(0), f0t ? T(0) : gsum, (lo2(accvd) + hi2(accvd)) * (quartic ? T(0.25) : T(0.5)),
                  T(0.5) * (lo2(accvi) + hi2(accvi))};
    finish_block(M, sc, A.partials, v, red, true);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// Box width: the whole row when N <= 256, else the largest divisor of N that is
// at most 256 elements and a multiple of 128 bytes (every box lands on a
// 128-byte boundary of its shared-memory row).
int box_width(int n, int esize)
{
    if (n <= 256) return n;
    for (int bw = 256; bw >= 1; bw--)
        if (n % bw == 0 && (bw * esize) % 16 == 0) return bw;
    return 0;
}

size_t smem_bytes(const TmaGeom& g, int esize)
{
    const size_t fslot = (size_t)2 * (g.ty + 3) * g.rs * g.nbx;
    const size_t pslot = (size_t)2 * (g.ty + 1) * g.rs * g.nbx;
    return 128 + g.rf * fslot + g.rp * pslot + 2 * pslot + (size_t)(g.rf + g.rp + 1) * 8 + 32 * kSums * 8;
}

int ipt_of(const TmaGeom& g) { return (g.items + kMaxThreads - 1) / kMaxThreads; }

// Resident blocks per SM of the kernel instance this geometry launches.
int occupancy(const TmaGeom& g, int esize, int threads, size_t smem)
{
    const void* fn = nullptr;
    const int ipt = ipt_of(g);
    if (esize == 4) fn = ipt == 1 ? (const void*)step_tma_kernel<float, 1> : ipt == 2 ? (const void*)step_tma_kernel<float, 2> : (const void*)step_tma_kernel<float, 3>;
    else fn = ipt == 1 ? (const void*)step_tma_kernel<double, 1> : ipt == 2 ? (const void*)step_tma_kernel<double, 2> : (const void*)step_tma_kernel<double, 3>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, threads, smem) != cudaSuccess) return 0;
    return blocks;
}

// Geometry for tile height ty, prefetch depth and `zr` planes of (y tile, z)
// work per block (0: one resident wave of persistent blocks).
bool make_geom(int n, int esize, int ty, int zr, int depth, TmaGeom* g, TmaConfig* cfg)
{
    const int vw = 16 / esize;
    if (n % 4 != 0 || n < 4 || ty < 1 || ty > n || n % ty != 0 || zr < 0 || depth < 1) return false;
    g->n = n; g->ty = ty; g->depth = depth;
    g->bw = box_width(n, esize);
    if (g->bw == 0) return false;
    g->nbx = n / g->bw;
    g->tall = (g->bw * esize) % 128 == 0 && ty + 3 <= 256;
    g->rs = ((g->bw * esize + 127) / 128) * 128;
    g->nyt = n / ty;
    g->rf = depth + 3;
    g->rp = depth + 1;
    g->items = 2 * (ty + 1) * (n / vw);
    const int ipt = ipt_of(*g);
    if (ipt > 3) return false;
    int threads = (g->items + ipt - 1) / ipt;
    threads = std::max(32, ((threads + 31) / 32) * 32);
    const size_t smem = smem_bytes(*g, esize);
    if (smem > 227 * 1024) return false;
    const int occ = occupancy(*g, esize, threads, smem);
    if (occ < 1) return false;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return false;
    const long long total = (long long)g->nyt * n;
    long long blocks;
    if (zr > 0) blocks = (total + zr - 1) / zr;
    else {
        blocks = (long long)sms * occ;
        if (total / blocks < 8) blocks = std::max(1LL, total / 8);   // keep runs of >= 8 planes
    }
    blocks = std::max(1LL, std::min(blocks, total));
    g->zr = (int)((total + blocks - 1) / blocks);
    cfg->ty = ty;
    cfg->zr = zr;
    cfg->depth = depth;
    cfg->threads = threads;
    cfg->smem = smem;
    cfg->blocks = (int)blocks;
    cfg->geom = *g;
    return true;
}

} // namespace

// Default geometry: the tallest tile (fewest redundant look-ahead rows and halo
// rows per owned row) whose ring fits with two planes in flight, else one.
bool tma_config(int n, int elem_bytes, int ty, int zr, TmaConfig* cfg)
{
    if (!encode_fn()) return false;
    TmaGeom g;
    const int depths[] = {2, 1};
    if (ty > 0) {
        for (int d : depths)
            if (make_geom(n, elem_bytes, ty, zr, d, &g, cfg)) return true;
        return false;
    }
    // prefer one vector per thread (no spills), then the tallest tile
    const int tys[] = {8, 4, 2, 1};
    for (int pass = 0; pass < 2; pass++)
        for (int t : tys) {
            if (n % t) continue;
            for (int d : depths) {
                TmaConfig c;
                if (!make_geom(n, elem_bytes, t, zr, d, &g, &c)) continue;
                if (pass == 0 && ipt_of(c.geom) > 1) continue;
                *cfg = c;
                return true;
            }
        }
    return false;
}

cudaError_t tma_encode_maps(const void* const ptrs[8], int n, int elem_bytes, int ty, void* out)
{
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const int bw = box_width(n, elem_bytes);
    if (bw == 0 || ty < 1) return cudaErrorInvalidValue;
    CUtensorMap* maps = (CUtensorMap*)out;
    for (int m = 0; m < kTmaMaps; m++) {
        const int i = m % 8;
        const bool momentum = (i % 4) >= 2;
        const int rows = m < 8 ? 1 : std::min(256, momentum ? ty + 1 : ty + 3);
        cuuint64_t dims[3] = {(cuuint64_t)n, (cuuint64_t)n, (cuuint64_t)n};
        cuuint64_t strides[2] = {(cuuint64_t)n * elem_bytes, (cuuint64_t)n * n * elem_bytes};
        cuuint32_t box[3] = {(cuuint32_t)bw, (cuuint32_t)std::min(rows, n), 1u};
        cuuint32_t estr[3] = {1u, 1u, 1u};
        CUresult r = enc(&maps[m], elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                         3, const_cast<void*>(ptrs[i]), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}

template <typename T>
cudaError_t launch_step_tma(const Bufs<T>& b, const Model& M, DevScalars* sc, double* partials,
                            const TmaConfig& cfg, const void* tmaps, cudaStream_t st)
{
    TmaArgs<T> A;
    std::memcpy(A.maps, tmaps, sizeof(A.maps));
    A.b = b;
    A.M = M;
    A.sc = sc;
    A.partials = partials;
    A.g = cfg.geom;
    if (A.g.n != M.n) return cudaErrorInvalidValue;
    const int ipt = (A.g.items + cfg.threads - 1) / cfg.threads;
    cudaError_t e;
    if (ipt <= 1) {
        e = cudaFuncSetAttribute(step_tma_kernel<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem);
        if (e != cudaSuccess) return e;
        step_tma_kernel<T, 1><<<cfg.blocks, cfg.threads, cfg.smem, st>>>(A);
    } else if (ipt == 2) {
        e = cudaFuncSetAttribute(step_tma_kernel<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem);
        if (e != cudaSuccess) return e;
        step_tma_kernel<T, 2><<<cfg.blocks, cfg.threads, cfg.smem, st>>>(A);
    } else if (ipt == 3) {
        e = cudaFuncSetAttribute(step_tma_kernel<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cfg.smem);
        if (e != cudaSuccess) return e;
        step_tma_kernel<T, 3><<<cfg.blocks, cfg.threads, cfg.smem, st>>>(A);
    } else {
        return cudaErrorInvalidConfiguration;
    }
    return cudaGetLastError();
}

template cudaError_t launch_step_tma<float>(const Bufs<float>&, const Model&, DevScalars*, double*,
                                            const TmaConfig&, const void*, cudaStream_t);
template cudaError_t launch_step_tma<double>(const Bufs<double>&, const Model&, DevScalars*, double*,
                                             const TmaConfig&, const void*, cudaStream_t);

} // namespace lat
