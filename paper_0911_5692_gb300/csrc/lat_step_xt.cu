// lat_step_xt.cu -- the fused 7-point leapfrog step on the plane ring with x
// tiles (variant 4), FP32 and FP64.
//
// Same step as the plane-ring kernel of lat_march.cuh (Sec. II.B, eq. evo with
// eq. scalar-evo; the sums of the new fields for eq. scale from the +y row and
// +z plane look-ahead; the FP64 a(t) update in the last block), with tiles that
// are narrower and taller: a block owns W columns (at most 32 or 16 16-byte
// vectors) of ty rows instead of full rows. Each staged row holds the tile's
// columns with one 16-byte vector on either side (periodic in x); the threads of
// those halo vectors stage them and kick and drift them too, so the new field
// one column right of the tile is at hand for the x differences of the sums.
// For wide lattices this trades a 16-byte halo per row for fewer halo and
// look-ahead rows per owned row (512^3 FP32: full rows allow only 4 owned rows
// per 7 staged).
#include <algorithm>

#include "lat_kernels.h"
#include "lat_march.cuh"

namespace lat {

namespace {

// March planes [z0, z0 + nz) of tile (xt, yt): W columns from x0 = xt W, ty rows
// from yt ty, through the ring S (the ring of lat_march.cuh over staged rows of
// W + 2 vectors).
template <typename T>
__device__ void march_segment_xt(const MarchLattice<T>& L, int xt, int W, int yt, int z0, int nz, T* S,
                                 MarchSums<T>& A, bool first)
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

    // the previous segment's last plane is read by every thread before the
    // prologue below refills the ring
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
    int sf = 0, sp = 0;

    for (int k = 0; k <= nz; k++) {
        const bool ahead = k == nz;
        const int z = z0 + k;
        cp_async_wait(D - 1);
        __syncthreads();
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
        // shuffles; rows that are only staged load harmlessly)
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
                PK<T>::ld(Ff - RW, up);
                PK<T>::ld(Ff + RW, dn);
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
                    // Laplacian as a sum of neighbour differences (exact for f = const + small)
                    const P lapu = add2(add2(add2(sub2(lft[v], c), sub2(rgt[v], c)),
                                             add2(sub2(up[v], c), sub2(dn[v], c))),
                                        add2(sub2(zm[v], c), sub2(zp[v], c)));
                    pn[f][v] = fma2(dtcl2, lapu, fma2(dtcf2, c, pv[v]));
                }
            }
            // potential part of the kick and the drift (lat_site.cuh)
#pragma unroll
            for (int v = 0; v < NP; v++) site_kick_drift<T>(L.K, cen[0][v], cen[1][v], pn[0][v], pn[1][v], g[0][v], g[1][v]);
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

        // sums over the owned sites of plane k-1 (x and y pairs, potential) and
        // the z pair (k-1, k), from the new fields written one plane ago
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
                    PK<T>::ld(Gf + RW, yn);
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
                        const P dxv = sub2(xn[v], gq[f][v]), dyv = sub2(yn[v], gq[f][v]),
                                dzv = sub2(g[f][v], gq[f][v]);
                        acc = fma2(dxv, dxv, fma2(dyv, dyv, fma2(dzv, dzv, acc)));
                    }
                    if (f == 0) A.accg0 = acc;
                    else A.accg1 = acc;
                }
#pragma unroll
                for (int v = 0; v < NP; v++) site_vsum<T>(L.K, gq[0][v], gq[1][v], A.accvd, A.accvi);
            }
        }
    }
}

struct ArgsXt {
    int ty, nyt, depth;
    int nxt, W;     // x tiles per row and their width
};

template <typename T, int MAXT>
__global__ void __launch_bounds__(MAXT, 1) step_xt_kernel(Bufs<T> B, Model M, DevScalars* sc, double* partials,
                                                          ArgsXt G)
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
    MarchSums<T> A;
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
        march_segment_xt(L, xt, G.W, yt, z0, nz, S, A, first);
    }
    T v[kSums];
    A.totals(L.K.quartic, v);
    finish_block(M, sc, partials, v, red, true);
}

constexpr int kMaxtsXt[] = {384, 512, 640, 768, 1024};

int maxt_xt_for(int threads)
{
    for (int m : kMaxtsXt)
        if (threads <= m) return m;
    return 0;
}

template <typename T>
const void* step_xt_fn(int maxt)
{
    switch (maxt) {
    case 384: return (const void*)step_xt_kernel<T, 384>;
    case 512: return (const void*)step_xt_kernel<T, 512>;
    case 640: return (const void*)step_xt_kernel<T, 640>;
    case 768: return (const void*)step_xt_kernel<T, 768>;
    default: return (const void*)step_xt_kernel<T, 1024>;
    }
}

size_t smem_xt(int rw, int esize, int ty, int depth)
{
    // the ring of lat_march.cuh over staged rows of rw elements
    return (size_t)esize * rw * ((depth + 3) * 2 * (ty + 3) + (depth + 1) * 2 * (ty + 1) + 2 * 2 * (ty + 1));
}

// x tiles per row: the fewest that keep a tile at most wmax vectors wide, among
// those that divide the row into whole vectors
int xt_tiles(int n, int vw, int wmax)
{
    const int q = n / vw;
    for (int nxt = (q + wmax - 1) / wmax; nxt <= q; nxt++)
        if (q % nxt == 0) return nxt;
    return q;
}

bool geom_xt(int n, int esize, int ty, int zr, int depth, MarchConfig* cfg)
{
    const int vw = 16 / esize;
    if (n % 4 != 0 || n < 4 || ty < 1 || ty > n || n % ty != 0) return false;
    if (depth < 1 || depth > 4) return false;
    // tiles of 32 vectors where a block of ty rows of them fits 1024 threads, else 16
    int nxt = xt_tiles(n, vw, 32);
    if ((ty + 3) * (n / nxt / vw + 2) > 1024) nxt = xt_tiles(n, vw, 16);
    const int W = n / nxt;
    int threads = (ty + 3) * (W / vw + 2);
    threads = ((threads + 31) / 32) * 32;
    if (threads > 1024) return false;
    const size_t smem = smem_xt(W + 2 * vw, esize, ty, depth);
    if (smem > 227 * 1024 - 2048) return false;
    const int maxt = maxt_xt_for(threads);
    const void* fn = esize == 4 ? step_xt_fn<float>(maxt) : step_xt_fn<double>(maxt);
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
    cfg->s27 = 0;
    cfg->xt = 1;
    cfg->nxt = nxt;
    return true;
}

} // namespace

bool xt_config(int n, int elem_bytes, int ty, int zr, int depth, MarchConfig* cfg)
{
    const int d = depth > 0 ? depth : 1;
    if (ty > 0) return geom_xt(n, elem_bytes, ty, zr, d, cfg);
    for (int t : {32, 16, 8, 4, 2, 1})
        if (geom_xt(n, elem_bytes, t, zr, d, cfg)) return true;
    return false;
}

template <typename T>
cudaError_t launch_step_xt(const Bufs<T>& b, const Model& M, DevScalars* sc, double* partials, const MarchConfig& cfg,
                           cudaStream_t st)
{
    ArgsXt G{cfg.ty, cfg.nyt, cfg.depth, cfg.nxt, M.n / cfg.nxt};
    switch (cfg.maxt) {
    case 384: step_xt_kernel<T, 384><<<cfg.blocks, cfg.threads, cfg.smem, st>>>(b, M, sc, partials, G); break;
    case 512: step_xt_kernel<T, 512><<<cfg.blocks, cfg.threads, cfg.smem, st>>>(b, M, sc, partials, G); break;
    case 640: step_xt_kernel<T, 640><<<cfg.blocks, cfg.threads, cfg.smem, st>>>(b, M, sc, partials, G); break;
    case 768: step_xt_kernel<T, 768><<<cfg.blocks, cfg.threads, cfg.smem, st>>>(b, M, sc, partials, G); break;
    default: step_xt_kernel<T, 1024><<<cfg.blocks, cfg.threads, cfg.smem, st>>>(b, M, sc, partials, G); break;
    }
    return cudaGetLastError();
}

template cudaError_t launch_step_xt<float>(const Bufs<float>&, const Model&, DevScalars*, double*, const MarchConfig&,
                                           cudaStream_t);
template cudaError_t launch_step_xt<double>(const Bufs<double>&, const Model&, DevScalars*, double*,
                                            const MarchConfig&, cudaStream_t);

} // namespace lat
