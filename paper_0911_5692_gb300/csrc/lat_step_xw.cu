// lat_step_xw.cu -- the compiled instances of the fused 7-point step over x
// tiles one warp wide (variant 5, lat_xw.cuh) for whole periodic lattices, and
// their launch configuration.
#include <algorithm>

#include "lat_xw.cuh"

namespace lat {

namespace {

// Compiled instances: (element bytes, N, TY, D).
struct XWKey {
    int esize, n, ty, depth;
};
constexpr XWKey kXW[] = {{4, 256, 16, 1}, {4, 256, 16, 2}, {4, 512, 16, 1}, {4, 512, 16, 2}, {4, 1024, 16, 1},
                         {8, 256, 16, 1}, {8, 512, 16, 1}};

template <typename T>
const void* xw_fn(int n, int ty, int depth, size_t* smem)
{
#define LAT_XW_CASE(NN, TT, DD)                                  \
    if (n == NN && ty == TT && depth == DD) {                    \
        *smem = xw::XW<T, NN, TT, DD, false>::SMEM;              \
        return (const void*)xw::step_xw_kernel<T, NN, TT, DD, false>; \
    }
    if constexpr (sizeof(T) == 4) {
        LAT_XW_CASE(256, 16, 1) LAT_XW_CASE(256, 16, 2) LAT_XW_CASE(512, 16, 1) LAT_XW_CASE(512, 16, 2)
        LAT_XW_CASE(1024, 16, 1)
    } else {
        LAT_XW_CASE(256, 16, 1) LAT_XW_CASE(512, 16, 1)
    }
#undef LAT_XW_CASE
    return nullptr;
}

const void* xw_kernel(int esize, int n, int ty, int depth, size_t* smem)
{
    for (const XWKey& k : kXW)
        if (k.esize == esize && k.n == n && k.ty == ty && k.depth == depth)
            return esize == 4 ? xw_fn<float>(n, ty, depth, smem) : xw_fn<double>(n, ty, depth, smem);
    return nullptr;
}

} // namespace

bool xw_config(int n, int elem_bytes, int ty, int zr, int depth, MarchConfig* cfg)
{
    const int tyv = ty > 0 ? ty : 16;
    // the instance with the requested depth, else any compiled depth (2 first:
    // two planes in flight measured 0.811-0.816 against 0.860 ms per step at
    // 512^3 FP32, 0.117 against 0.124 ms at 256^3)
    int d = depth;
    size_t smem = 0;
    const void* fn = nullptr;
    if (d > 0) fn = xw_kernel(elem_bytes, n, tyv, d, &smem);
    else
        for (int dd : {2, 1})
            if ((fn = xw_kernel(elem_bytes, n, tyv, dd, &smem))) {
                d = dd;
                break;
            }
    if (!fn || smem > 227 * 1024 - 2048) return false;
    const int vw = 16 / elem_bytes, w = 32 * vw, nxt = n / w;
    const int threads = (tyv + 4) * 32;
    if (allow_dynamic_smem(fn, smem) != cudaSuccess) return false;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem) != cudaSuccess || occ < 1) return false;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return false;
    const int nyt = n / tyv;
    const long long tiles = (long long)nyt * nxt, units = tiles * n;
    long long blocks = 0;
    // whole groups of nxt blocks (the x tiles of a y tile, marching together)
    if (zr > 0) blocks = tiles * ((n + std::min(zr, n) - 1) / std::min(zr, n));
    else blocks = std::min((long long)sms * occ, units) / nxt * nxt;
    const long long groups = blocks / nxt;
    cfg->ty = tyv;
    // planes of the first group's first run (the z chunk of one tile when the
    // groups march the tiles in step, lat_layout.cuh)
    const Layout L0 = tile_layout(nyt, (int)groups, 0, n);
    cfg->zr = std::min(L0.uend - L0.ubeg, L0.zspan);
    cfg->nzc = (int)((groups + nyt - 1) / nyt);
    cfg->depth = d;
    cfg->threads = threads;
    cfg->maxt = threads;
    cfg->fast = 1;
    cfg->smem = smem;
    cfg->nyt = nyt;
    cfg->blocks = (int)blocks;
    cfg->nzl = 0;
    cfg->zbase = 0;
    cfg->s27 = 0;
    cfg->xt = 0;
    cfg->xw = 1;
    cfg->nxt = nxt;
    return true;
}

template <typename T>
cudaError_t launch_step_xw(const Bufs<T>& b, const Model& M, DevScalars* sc, double* partials, const MarchConfig& cfg,
                           cudaStream_t st)
{
    size_t smem = 0;
    const void* fn = xw_fn<T>(M.n, cfg.ty, cfg.depth, &smem);
    if (!fn) return cudaErrorInvalidValue;
    xw::SlabRun R{0, 0, nullptr};
    void* args[] = {(void*)&b, (void*)&M, (void*)&sc, (void*)&partials, (void*)&R};
    return cudaLaunchKernel(fn, dim3(cfg.blocks), dim3(cfg.threads), args, cfg.smem, st);
}

template cudaError_t launch_step_xw<float>(const Bufs<float>&, const Model&, DevScalars*, double*, const MarchConfig&,
                                           cudaStream_t);
template cudaError_t launch_step_xw<double>(const Bufs<double>&, const Model&, DevScalars*, double*,
                                            const MarchConfig&, cudaStream_t);

} // namespace lat
