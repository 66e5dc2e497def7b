// lat_step_march.cu -- the fused leapfrog step on a shared-memory plane ring,
// for any lattice side and tile height (FP32 and FP64).
//
// The step (Sec. II.B, eq. evo with eq. scalar-evo: 7-point Laplacian,
// potential derivative, kick and drift of both fields; the sums of the new
// fields for eq. scale from a one-site look-ahead rim; the FP64 a(t) update in
// the last block), laid out for the GB300 memory system. The z-march segment
// itself (ring, asynchronous copies, look-ahead rim) is in lat_march.cuh.
// Per-thread asynchronous copies keep enough bytes moving per SM to run near
// the HBM rate on this access pattern; a ring filled by a few large TMA boxes
// per block measured well below it and was not kept. One persistent wave of
// blocks shares the (y tile, z plane) units evenly. This file also holds the
// launch dispatch of every step kernel (launch_step_march) and the process-wide
// shared-memory opt-in (allow_dynamic_smem).
#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include "lat_kernels.h"
#include "lat_march.cuh"

namespace lat {

cudaError_t allow_dynamic_smem(const void* fn, size_t bytes)
{
    static std::mutex mx;
    static std::map<std::pair<int, const void*>, size_t> granted;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mx);
    size_t& g = granted[{dev, fn}];
    if (bytes <= g) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) g = bytes;
    return e;
}


namespace {

struct MarchArgs {
    int ty, nzc, nyt, depth;
    int nzl;        // planes of the z domain: n, or the owned planes of a z-slab
    int zbase;      // slab: stored plane of z = z + zbase (0 when periodic)
    int periodic;   // 1: periodic z (a whole lattice); 0: z-slab with halo planes
};

template <typename T, int MAXT, bool SPLIT>
__global__ void __launch_bounds__(MAXT, (MAXT <= 512 ? 2 : 1))
    step_march_kernel(Bufs<T> B, Model M, DevScalars* sc, double* partials, MarchArgs G, double* sums_out)
{
    __shared__ double red[32 * kSums];
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (sc->status != LAT_OK) return;
    T* const S = reinterpret_cast<T*>(smem_raw);
    const int n = M.n;

    // ping-pong parity; buffers are selected with constant indices (a runtime
    // index into the parameter block would copy it to local memory)
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
    L.periodic = G.periodic != 0;
    L.zbase = G.zbase;
    MarchSums<T> A;
    A.zero();

    // Work: the nyt * nzl (y tile, z plane) units in tile-major order; block b
    // takes units [b U / B, (b+1) U / B) and marches them as one segment per y
    // tile it touches (B = nyt * c gives c balanced z chunks per tile).
    const int nzl = G.nzl;
    const long long U = (long long)G.nyt * nzl;
    long long u = (long long)blockIdx.x * U / gridDim.x;
    const long long uend = ((long long)blockIdx.x + 1) * U / gridDim.x;
    for (bool first = true; u < uend; first = false) {
        const int yt = (int)(u / nzl);
        const int z0 = (int)(u - (long long)yt * nzl);
        const int nz = (int)min((long long)(nzl - z0), uend - u);
        u += nz;
        march_segment<T, SPLIT>(L, yt, z0, nz, S, A, first);
    }
    T v[kSums];
    A.totals(L.K.quartic, v);
    if (sums_out) finish_block_sums(M, sc, partials, v, red, sums_out);
    else finish_block(M, sc, partials, v, red, true);
}


// launch-bound instances: the register budget follows the block size
constexpr int kMaxts[] = {448, 512, 704, 768, 896, 1024};
int maxt_for(int threads)
{
    for (int m : kMaxts)
        if (threads <= m) return m;
    return 0;
}

// the instance for a block size; `split`: the lattice stores phi split
template <typename T>
const void* march_fn(int maxt, bool split)
{
#define LAT_MARCH_FN(MT) \
    return split ? (const void*)step_march_kernel<T, MT, true> : (const void*)step_march_kernel<T, MT, false>
    switch (maxt) {
    case 448: LAT_MARCH_FN(448);
    case 512: LAT_MARCH_FN(512);
    case 704: LAT_MARCH_FN(704);
    case 768: LAT_MARCH_FN(768);
    case 896: LAT_MARCH_FN(896);
    default: LAT_MARCH_FN(1024);
    }
#undef LAT_MARCH_FN
}

// the dynamic shared memory opt-in for both instances of a block size
bool march_smem_attr(int esize, int maxt, size_t smem)
{
    for (bool split : {false, true}) {
        const void* fn = esize == 4 ? march_fn<float>(maxt, split) : march_fn<double>(maxt, split);
        if (allow_dynamic_smem(fn, smem) != cudaSuccess) return false;
    }
    return true;
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
    const void* fn = fast ? fast : esize == 4 ? march_fn<float>(maxt, true) : march_fn<double>(maxt, true);
    if (fast ? allow_dynamic_smem(fn, smem) != cudaSuccess : !march_smem_attr(esize, maxt, smem))
        return false;
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
bool march_slab_config(int n, int elem_bytes, int nzl, MarchConfig* cfg)
{
    if (nzl < 1) return false;
    const int vw = 16 / elem_bytes;
    for (int ty : {16, 8, 4, 2, 1}) {
        if (ty > n || n % ty != 0) continue;
        int threads = ((ty + 3) * (n / vw) + 31) / 32 * 32;
        if (threads > 1024) continue;
        const size_t smem = march_smem(n, elem_bytes, ty, 1);
        if (smem > 227 * 1024 - 2048) continue;
        const int maxt = maxt_for(threads);
        const void* fn = elem_bytes == 4 ? march_fn<float>(maxt, true) : march_fn<double>(maxt, true);
        if (!march_smem_attr(elem_bytes, maxt, smem)) continue;
        int occ = 0, dev = 0, sms = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem) != cudaSuccess || occ < 1) continue;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return false;
        const long long units = (long long)(n / ty) * nzl;
        const long long blocks = std::min<long long>((long long)sms * occ, units);
        cfg->ty = ty;
        cfg->zr = (int)((units + blocks - 1) / blocks);
        cfg->nzc = 0;
        cfg->depth = 1;
        cfg->threads = threads;
        cfg->maxt = maxt;
        cfg->fast = 0;
        cfg->smem = smem;
        cfg->nyt = n / ty;
        cfg->blocks = (int)blocks;
        cfg->nzl = nzl;
        cfg->zbase = 1;
        return true;
    }
    return false;
}

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
                              const MarchConfig& cfg, cudaStream_t st, double* sums_out)
{
    if (cfg.s27) {
        if (sums_out || cfg.nzl) return cudaErrorInvalidValue;
        return cfg.xw ? launch_step27w<T>(b, M, sc, partials, cfg, st) : launch_step27<T>(b, M, sc, partials, cfg, st);
    }
    if (cfg.xt) {
        if (sums_out || cfg.nzl) return cudaErrorInvalidValue;
        return launch_step_xt<T>(b, M, sc, partials, cfg, st);
    }
    if (cfg.xw) {
        if (sums_out || cfg.nzl) return cudaErrorInvalidValue;
        return launch_step_xw<T>(b, M, sc, partials, cfg, st);
    }
    if (cfg.fast && !sums_out && cfg.nzl == 0) return launch_step_fast<T>(b, M, sc, partials, cfg, st);
    MarchArgs G{cfg.ty, cfg.nzc, cfg.nyt, cfg.depth, cfg.nzl > 0 ? cfg.nzl : M.n, cfg.zbase, cfg.nzl > 0 ? 0 : 1};
    double* so = sums_out;
    const void* fn = march_fn<T>(cfg.maxt, M.split != 0);
    void* args[] = {(void*)&b, (void*)&M, (void*)&sc, (void*)&partials, (void*)&G, (void*)&so};
    cudaError_t e = cudaLaunchKernel(fn, dim3(cfg.blocks), dim3(cfg.threads), args, cfg.smem, st);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template cudaError_t launch_step_march<float>(const Bufs<float>&, const Model&, DevScalars*, double*,
                                              const MarchConfig&, cudaStream_t, double*);
template cudaError_t launch_step_march<double>(const Bufs<double>&, const Model&, DevScalars*, double*,
                                               const MarchConfig&, cudaStream_t, double*);

} // namespace lat
