// lat_step_march.cu -- the fast fused leapfrog step (FP32 and FP64).
//
// Same step as lat_step_simple.cu (Sec. II.B, eq. evo with eq. scalar-evo:
// 7-point Laplacian, potential derivative, kick and drift of both fields; the
// sums of the new fields for eq. scale from a one-site look-ahead rim; the FP64
// a(t) update in the last block), laid out for the GB300 memory system.
//
// A block owns full x rows, `ty` rows in y and a chunk of `zr` planes in z, and
// marches the chunk in +z as the paper's Fig. 1 kernel does. One thread owns one
// 16-byte vector (4 floats or 2 doubles) of one row of the tile or of its halo
// (one row below, two above: the second for the look-ahead rim). Planes are
// staged in a shared-memory ring by per-thread 16-byte asynchronous copies
// (cp.async) issued one plane ahead: every thread keeps its own copies in flight,
// which is what keeps enough bytes moving per SM to run at the HBM rate on this
// access pattern (a ring filled by a few large TMA boxes per block measured
// well below it; that variant is kept in lat_step_tma.cu), and no registers are
// spent on staging. One barrier per plane: the copies for the next plane are
// issued right after it into the slots the previous plane has released.
//
// FP32 arithmetic is done on packed f32x2 pairs. The forward differences of the
// new fields in x and y, and their potential, are summed one plane later from
// a double-buffered shared copy of the new fields; the z difference uses the
// previous plane's new fields. Sums accumulate in FP32 per thread and FP64 per
// block.
#include <algorithm>

#include "lat_kernels.h"
#include "lat_async.cuh"
#include "lat_pairs.cuh"

namespace lat {

namespace {



struct MarchArgs {
    int ty, nzc, nyt, depth;
};

// Shared ring of the march for prefetch depth D: D+3 field-plane slots
// [slot][field][ty+3 rows][n] (planes z-1, z, z+1 in use, D planes in flight),
// D+1 momentum slots [slot][field][ty+1 rows][n], 2 new-field planes
// [buf][field][ty+1 rows][n]. Offsets in elements.
struct RingGeom {
    uint32_t fieldF, slotF, fieldP, slotP, fieldG, planeG, p0, g0;
    int rf, rp;
};

__device__ __forceinline__ RingGeom ring_geom(int n, int ty, int depth)
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

template <typename T, int MAXT>
__global__ void __launch_bounds__(MAXT, (MAXT <= 512 ? 2 : 1)) step_march_kernel(Bufs<T> B, Model M, DevScalars* sc, double* partials,
                                                          MarchArgs G)
{
    typedef typename PK<T>::P P;
    constexpr int NP = PK<T>::NP;
    constexpr int VW = 2 * NP;
    __shared__ double red[32 * kSums];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (sc->status != LAT_OK) return;
    T* const S = reinterpret_cast<T*>(smem_raw);

    const int n = M.n, ty = G.ty, Q = n / VW;
    const int t = threadIdx.x;
    const int rho_raw = t / Q;
    const bool live = rho_raw < ty + 3;                 // threads past the tile only join the barriers
    const int rho = min(rho_raw, ty + 2);
    const int x = live ? (t - rho_raw * Q) * VW : 0;
    const bool comp = live && rho >= 1 && rho <= ty + 1;   // computes a new vector (owned rows + look-ahead row)
    const bool own = live && rho >= 1 && rho <= ty;
    const int dl = x == 0 ? n - 1 : -1;                     // left neighbour of the first site (periodic)
    const int dr = x + VW == n ? VW - n : VW;                // right neighbour of the last site
    const int D = G.depth;
    const RingGeom R = ring_geom(n, ty, D);
    const uint32_t offF = (uint32_t)rho * n + x;            // this vector in a field plane
    const uint32_t offP = (uint32_t)(comp ? rho - 1 : 0) * n + x;   // in a momentum / new-field plane

    // Work: the nyt * n (y tile, z plane) units in tile-major order; block b
    // takes units [b U / B, (b+1) U / B) and marches them as one segment per y
    // tile it touches (B = nyt * c gives c balanced z chunks per tile).
    const long long U = (long long)G.nyt * n;
    long long u = (long long)blockIdx.x * U / gridDim.x;
    const long long uend = ((long long)blockIdx.x + 1) * U / gridDim.x;
    int z0 = 0, nz = 0;
    uint32_t rowg = 0;
    const uint32_t nn = (uint32_t)n * n;
    // ping-pong parity; buffers are selected with constant indices (a runtime
    // index into the parameter block would copy it to local memory)
    const bool par = (sc->step & 1) != 0;
    const T* const f0 = par ? B.f[1][0] : B.f[0][0];
    const T* const f1 = par ? B.f[1][1] : B.f[0][1];
    const T* const p0 = par ? B.p[1][0] : B.p[0][0];
    const T* const p1 = par ? B.p[1][1] : B.p[0][1];

    // f' += dt (cL Lap f + cF f - dV/df), f += dt f', with the 1/dx^2 of the
    // Laplacian folded into dt cL
    const T dt_s = step_coef<T>(sc, 4);
    const T dtcl = step_coef<T>(sc, 0), dtcf = step_coef<T>(sc, 1);
    const T mdtcdom = step_coef<T>(sc, 2), mdtkap = step_coef<T>(sc, 3);
    const bool quartic = M.beta == 4;
    P accg0 = mk2(T(0), T(0)), accg1 = accg0, accvd = accg0, accvi = accg0;

    // copies of this thread's vectors of plane z0 + zrel: f into field slot
    // (zrel + 1) mod (D+3), momenta into momentum slot zrel mod (D+1); the slot
    // is passed in (kept as running counters, no division in the loop)
    auto fetch_f = [&](int zrel, int slot) {          // zrel in [-1, nz + 1]
        const uint32_t gi = (uint32_t)wrapn(z0 + zrel, n) * nn + rowg;
        T* d = S + (uint32_t)slot * R.slotF + offF;
        cp_async16(d, f0 + gi);
        cp_async16(d + R.fieldF, f1 + gi);
    };
    auto fetch_p = [&](int zrel, int slot) {          // zrel in [0, nz]
        const uint32_t gi = (uint32_t)wrapn(z0 + zrel, n) * nn + rowg;
        T* d = S + R.p0 + (uint32_t)slot * R.slotP + offP;
        cp_async16(d, p0 + gi);
        cp_async16(d + R.fieldP, p1 + gi);
    };
    // x neighbours in the adjacent lanes (same row, not wrapped), else shared memory
    const int lane = t & 31;
    const int qv = x / VW;
    const bool nbl = qv > 0 && lane > 0, nbr = qv < Q - 1 && lane < 31;
    auto addm = [](int a, int b, int m) { return a + b >= m ? a + b - m : a + b; };

    for (bool first = true; u < uend; first = false) {
        const int yt = (int)(u / n);
        z0 = (int)(u - (long long)yt * n);
        nz = (int)min((long long)(n - z0), uend - u);
        u += nz;
        rowg = (uint32_t)wrapn(yt * ty - 1 + rho, n) * n + x;
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
                    const P dtcl2 = mk2(dtcl, dtcl), dtcf2 = mk2(dtcf, dtcf);
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
                const P mdtcdom2 = mk2(mdtcdom, mdtcdom), mdtkap2 = mk2(mdtkap, mdtkap), dt2 = mk2(dt_s, dt_s);
#pragma unroll
                for (int v = 0; v < NP; v++) {
                    // potential: f0 gets -dt (cdom f0^(beta-1) + kappa f0 f1^2), f1 gets -dt kappa f0^2 f1
                    const P a0 = cen[0][v], a1 = cen[1][v];
                    const P a0a1 = mul2(a0, a1);
                    const P dom = quartic ? mul2(mul2(a0, a0), a0) : a0;
                    pn[0][v] = fma2(mdtcdom2, dom, fma2(mdtkap2, mul2(a0a1, a1), pn[0][v]));
                    pn[1][v] = fma2(mdtkap2, mul2(a0a1, a0), pn[1][v]);
                    g[0][v] = fma2(dt2, pn[0][v], a0);
                    g[1][v] = fma2(dt2, pn[1][v], a1);
                }
                if (!ahead) {
                    if (own) {
                        const uint32_t gi = (uint32_t)z * nn + rowg;
                        PK<T>::st((par ? B.p[0][0] : B.p[1][0]) + gi, pn[0]);
                        PK<T>::st((par ? B.p[0][1] : B.p[1][1]) + gi, pn[1]);
                        PK<T>::st((par ? B.f[0][0] : B.f[1][0]) + gi, g[0]);
                        PK<T>::st((par ? B.f[0][1] : B.f[1][1]) + gi, g[1]);
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
                    P acc = f == 0 ? accg0 : accg1;
#pragma unroll
                    for (int v = 0; v < NP; v++) {
                        const P dxv = sub2(xn[v], gq[f][v]), dyv = sub2(yn[v], gq[f][v]), dzv = sub2(g[f][v], gq[f][v]);
                        acc = fma2(dxv, dxv, fma2(dyv, dyv, fma2(dzv, dzv, acc)));
                    }
                    if (f == 0) accg0 = acc;
                    else accg1 = acc;
                }
#pragma unroll
                for (int v = 0; v < NP; v++) {
                    const P sq = mul2(gq[0][v], gq[0][v]);
                    accvd = quartic ? fma2(sq, sq, accvd) : add2(sq, accvd);
                    accvi = fma2(sq, mul2(gq[1][v], gq[1][v]), accvi);
                }
                }
            }
        }
    } // segments

    // per-thread sums in the element type (the 1/beta and 1/2 factors are
    // powers of two, exact); the block folds them as finish_block describes
    T v[kSums] = {lo2(accg0) + hi2(accg0), lo2(accg1) + hi2(accg1),
                  (lo2(accvd) + hi2(accvd)) * (quartic ? T(0.25) : T(0.5)),
                  T(0.5) * (lo2(accvi) + hi2(accvi))};
    finish_block(M, sc, partials, v, red, true);
}

// launch-bound instances: the register budget follows the block size
constexpr int kMaxts[] = {448, 512, 704, 768, 896, 1024};
int maxt_for(int threads)
{
    for (int m : kMaxts)
        if (threads <= m) return m;
    return 0;
}

template <typename T>
const void* march_fn(int maxt)
{
    switch (maxt) {
    case 448: return (const void*)step_march_kernel<T, 448>;
    case 512: return (const void*)step_march_kernel<T, 512>;
    case 704: return (const void*)step_march_kernel<T, 704>;
    case 768: return (const void*)step_march_kernel<T, 768>;
    case 896: return (const void*)step_march_kernel<T, 896>;
    default: return (const void*)step_march_kernel<T, 1024>;
    }
}

size_t march_smem(int n, int esize, int ty, int depth)
{
    // depth+3 field-plane slots, depth+1 momentum slots, 2 new-field planes (both fields each)
    return (size_t)esize * n * ((depth + 3) * 2 * (ty + 3) + (depth + 1) * 2 * (ty + 1) + 2 * 2 * (ty + 1));
}

bool march_geom(int n, int esize, int ty, int zr, int depth, MarchConfig* cfg)
{
    const int vw = 16 / esize;
    if (n % 4 != 0 || n < 4 || ty < 1 || ty > n || n % ty != 0) return false;
    int threads = (ty + 3) * (n / vw);
    threads = ((threads + 31) / 32) * 32;
    if (threads > 1024) return false;
    if (depth < 1 || depth > 4) return false;
    size_t fast_smem = 0;
    const void* fast = fast_kernel(esize, n, ty, depth, &fast_smem);
    const size_t smem = fast ? fast_smem : march_smem(n, esize, ty, depth);
    if (smem > 227 * 1024 - 2048) return false;   // the opt-in limit less the static arrays
    const int maxt = maxt_for(threads);
    const void* fn = fast ? fast : esize == 4 ? march_fn<float>(maxt) : march_fn<double>(maxt);
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return false;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem) != cudaSuccess || occ < 1) return false;
    // blocks: for a requested z length zr, nyt * ceil(n / zr) blocks (balanced
    // z chunks of each y tile); else one resident wave, each block taking an
    // equal share of the (y tile, z plane) units
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return false;
    const long long slots = (long long)sms * occ;
    const int nyt = n / ty;
    const long long units = (long long)nyt * n;
    long long blocks = 0;
    if (zr > 0) blocks = (long long)nyt * ((n + std::min(zr, n) - 1) / std::min(zr, n));
    else blocks = std::min(slots, units);
    cfg->ty = ty;
    cfg->zr = (int)((units + blocks - 1) / blocks);
    cfg->nzc = (int)((blocks + nyt - 1) / nyt);
    cfg->depth = depth;
    cfg->threads = threads;
    cfg->maxt = maxt;
    cfg->fast = fast ? 1 : 0;
    cfg->smem = smem;
    cfg->nyt = nyt;
    cfg->blocks = (int)blocks;
    return true;
}

} // namespace

// Default geometry: the tallest tile (fewest halo and look-ahead rows per owned
// row) whose block fits in 1024 threads.
bool march_config(int n, int elem_bytes, int ty, int zr, int depth, MarchConfig* cfg)
{
    const int d = depth > 0 ? depth : 1;
    if (ty > 0) return march_geom(n, elem_bytes, ty, zr, d, cfg);
    const int tys[] = {16, 8, 4, 2, 1};
    for (int t : tys)
        if (march_geom(n, elem_bytes, t, zr, d, cfg)) return true;
    return false;
}

template <typename T>
cudaError_t launch_step_march(const Bufs<T>& b, const Model& M, DevScalars* sc, double* partials,
                              const MarchConfig& cfg, cudaStream_t st)
{
    if (cfg.fast) return launch_step_fast<T>(b, M, sc, partials, cfg, st);
    MarchArgs G{cfg.ty, cfg.nzc, cfg.nyt, cfg.depth};
    switch (cfg.maxt) {
    case 448: step_march_kernel<T, 448><<<cfg.blocks, cfg.threads, cfg.smem, st>>>(b, M, sc, partials, G); break;
    case 512: step_march_kernel<T, 512><<<cfg.blocks, cfg.threads, cfg.smem, st>>>(b, M, sc, partials, G); break;
    case 704: step_march_kernel<T, 704><<<cfg.blocks, cfg.threads, cfg.smem, st>>>(b, M, sc, partials, G); break;
    case 768: step_march_kernel<T, 768><<<cfg.blocks, cfg.threads, cfg.smem, st>>>(b, M, sc, partials, G); break;
    case 896: step_march_kernel<T, 896><<<cfg.blocks, cfg.threads, cfg.smem, st>>>(b, M, sc, partials, G); break;
    default: step_march_kernel<T, 1024><<<cfg.blocks, cfg.threads, cfg.smem, st>>>(b, M, sc, partials, G); break;
    }
    return cudaGetLastError();
}

template cudaError_t launch_step_march<float>(const Bufs<float>&, const Model&, DevScalars*, double*,
                                              const MarchConfig&, cudaStream_t);
template cudaError_t launch_step_march<double>(const Bufs<double>&, const Model&, DevScalars*, double*,
                                               const MarchConfig&, cudaStream_t);

} // namespace lat
