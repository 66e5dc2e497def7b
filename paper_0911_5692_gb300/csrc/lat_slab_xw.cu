// lat_slab_xw.cu -- the fused 7-point step over x tiles one warp wide (lat_xw.cuh)
// for a range of a z-slab's owned planes: the compiled instances, their launch
// configuration and launch.
#include <algorithm>

#include "lat_xw.cuh"

namespace lat {

namespace {

template <typename T>
const void* slab_xw_fn(int n, size_t* smem, int* depth)
{
#define LAT_SLAB_XW_CASE(NN, DD)                                              \
    if (n == NN) {                                                            \
        *depth = DD;                                                          \
        *smem = xw::XW<T, NN, 16, DD, true>::SMEM;                            \
        return (const void*)xw::step_xw_kernel<T, NN, 16, DD, true>;          \
    }
    // two planes in flight for FP32 (as the whole-lattice default), one for FP64
    if constexpr (sizeof(T) == 4) {
        LAT_SLAB_XW_CASE(256, 2) LAT_SLAB_XW_CASE(512, 2)
    } else {
        LAT_SLAB_XW_CASE(256, 1)
    }
#undef LAT_SLAB_XW_CASE
    return nullptr;
}

} // namespace

bool slab_xw_config(int n, int elem_bytes, int nz, MarchConfig* cfg)
{
    if (nz < 1) return false;
    size_t smem = 0;
    int d = 1;
    const void* fn = elem_bytes == 4 ? slab_xw_fn<float>(n, &smem, &d) : slab_xw_fn<double>(n, &smem, &d);
    if (!fn || smem > 227 * 1024 - 2048) return false;
    constexpr int ty = 16;
    const int vw = 16 / elem_bytes, w = 32 * vw, nxt = n / w;
    const int threads = (ty + 4) * 32;
    if (allow_dynamic_smem(fn, smem) != cudaSuccess) return false;
    int occ = 0, dev = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, threads, smem) != cudaSuccess || occ < 1) return false;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) return false;
    const int nyt = n / ty;
    const long long units = (long long)nyt * nz;
    // whole groups of nxt blocks, at most one resident wave, at most one unit per group
    const long long groups = std::max<long long>(1, std::min<long long>((long long)sms * occ / nxt, units));
    cfg->ty = ty;
    cfg->zr = (int)((units + groups - 1) / groups);
    cfg->nzc = 0;
    cfg->depth = d;
    cfg->threads = threads;
    cfg->maxt = threads;
    cfg->fast = 1;
    cfg->smem = smem;
    cfg->nyt = nyt;
    cfg->blocks = (int)(groups * nxt);
    cfg->nzl = nz;
    cfg->zbase = 1;
    cfg->s27 = 0;
    cfg->xt = 0;
    cfg->xw = 1;
    cfg->nxt = nxt;
    return true;
}

template <typename T>
cudaError_t launch_slab_xw(const xw::SlabRun& R, const Model& M, DevScalars* sc, double* partials,
                           const MarchConfig& cfg, cudaStream_t st)
{
    size_t smem = 0;
    int d = 1;
    const void* fn = slab_xw_fn<T>(M.n, &smem, &d);
    if (!fn || !R.sums_out || d != cfg.depth || R.nranges < 1 || R.nranges > xw::kMaxSlabRanges)
        return cudaErrorInvalidValue;
    const Bufs<T> unused{};
    void* args[] = {(void*)&unused, (void*)&M, (void*)&sc, (void*)&partials, (void*)&R};
    return cudaLaunchKernel(fn, dim3(cfg.blocks), dim3(cfg.threads), args, cfg.smem, st);
}

template cudaError_t launch_slab_xw<float>(const xw::SlabRun&, const Model&, DevScalars*, double*, const MarchConfig&,
                                           cudaStream_t);
template cudaError_t launch_slab_xw<double>(const xw::SlabRun&, const Model&, DevScalars*, double*,
                                            const MarchConfig&, cudaStream_t);

} // namespace lat
