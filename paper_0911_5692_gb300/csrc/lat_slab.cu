// lat_slab.cu -- one lattice split into z-slabs, one slab per handle (the
// multi-GPU form the paper leaves as future work, Sec. IV).
//
// A slab handle owns planes [z0, z0 + nzl) of an N^3 lattice. Its eight arrays
// hold nzl + 3 planes each: stored plane p is global plane z0 - 1 + p (mod N),
// so p = 0 is the halo below, 1 .. nzl the owned planes and nzl + 1, nzl + 2
// the halos above (the second for the look-ahead rim of the step's sums).
// One step of the whole lattice is then, per slab:
//   1. halo exchange (by the caller): f planes 0, nzl+1, nzl+2 and pi plane
//      nzl+1 of the current ping-pong set from the neighbouring slabs;
//   2. lat_slab_step: the fused step (Sec. II.B, eq. evo with eq. scalar-evo) on
//      the owned planes, writing the slab's share of the volume averages of the
//      new fields (sums over its sites / N^3);
//   3. the shares of all slabs added (an allreduce of four FP64 numbers);
//   4. lat_slab_advance: the FP64 scale-factor update (eq. scale) from the
//      total, identical on every slab.
// Before the first step, lat_slab_sums + lat_slab_advance(advance = 0) set the
// coefficients from the starting fields.
//
// Step 2 may be taken in z ranges (lat_slab_step_range), each writing its own
// shares: owned planes 2 .. nzl - 3 read no halo plane (their runs end on the
// look-ahead plane nzl - 2, whose z neighbours are owned), so they can run while
// the halos are still in flight; planes 0, 1 and nzl - 2, nzl - 1 follow once
// the halos are in, and are the planes the neighbours need for the next step.
// Slabs of one lattice held by one process (one GPU) can take step 2 in one
// launch over ranges of all of them (lat_slab_step_ranges), copy their halos in
// one launch (lat_copy_regions) and take steps 3 and 4 in one launch
// (lat_slab_advance_local).
#include <algorithm>
#include <cstdint>

#include "lat_internal.h"
#include "lat_site.cuh"

namespace lat {

namespace {

// Shares of the four volume averages of the current fields over the owned
// sites (forward differences; the +z neighbour of the top plane is the halo).
template <typename T>
__global__ void __launch_bounds__(256) slab_sums_kernel(Bufs<T> B, Model M, DevScalars* sc, double* partials,
                                                        int nzl, double* sums_out)
{
    __shared__ double red[32 * kSums];
    const int n = M.n;
    const int par = (int)(sc->step & 1);
    const T* __restrict__ f0 = par ? B.f[1][0] : B.f[0][0];
    const T* __restrict__ f1 = par ? B.f[1][1] : B.f[0][1];
    const bool quartic = M.beta == 4;
    const double P = sc->bgf, vfac = site_vsum_factor<double>(quartic);
    double acc[kSums] = {0.0, 0.0, 0.0, 0.0};
    const size_t nn = (size_t)n * n;
    const long long cols = (long long)n * n;
    for (long long col = (long long)blockIdx.x * blockDim.x + threadIdx.x; col < cols;
         col += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(col % n), y = (int)(col / n);
        const int xp = x == n - 1 ? 0 : x + 1, yp = y == n - 1 ? 0 : y + 1;
        for (int z = 0; z < nzl; z++) {
            const size_t pl = (size_t)(z + 1) * nn, pu = (size_t)(z + 2) * nn;
            const size_t c = pl + (size_t)y * n + x;
            const double a0 = (double)f0[c], a1 = (double)f1[c];
            const double e0 = (double)f0[pl + (size_t)y * n + xp] - a0, e1 = (double)f0[pl + (size_t)yp * n + x] - a0,
                         e2 = (double)f0[pu + (size_t)y * n + x] - a0;
            const double h0 = (double)f1[pl + (size_t)y * n + xp] - a1, h1 = (double)f1[pl + (size_t)yp * n + x] - a1,
                         h2 = (double)f1[pu + (size_t)y * n + x] - a1;
            acc[0] += e0 * e0 + e1 * e1 + e2 * e2;
            acc[1] += h0 * h0 + h1 * h1 + h2 * h2;
            // potential terms about the homogeneous mode (lat_site.cuh)
            acc[2] += vfac * vdiff_dom(a0, P, P * P, quartic);
            acc[3] += 0.5 * vint(a0, a1, P);
        }
    }
    finish_block_sums(M, sc, partials, acc, red, sums_out);
}

// The scalars after one step (or, advance = 0, the coefficients of the first
// step) from the total of all slabs' shares.
__global__ void slab_advance_kernel(Model M, DevScalars* sc, const double* sums, int advance)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    DevScalars s = *sc;
    if (s.status != LAT_OK) return;
    const double S[kSums] = {sums[0], sums[1], sums[2], sums[3]};
    advance_scalars(M, s, S, advance != 0);
    s.ticket = 0u;
    *sc = s;
}

// The scalars of every slab of a lattice held by this process after one step
// (advance = 0: the coefficients of the first step), in one launch: each thread
// adds the shares in the order given (so every slab sees the same total, bit
// for bit, as after an allreduce in that order) and advances its own slab.
constexpr int kMaxLocalSlabs = 64, kMaxLocalShares = 192;

struct LocalAdvance {
    DevScalars* sc[kMaxLocalSlabs];
    const double* share[kMaxLocalShares];
};

__global__ void slab_advance_local_kernel(Model M, LocalAdvance A, int nslabs, int nshares, int advance)
{
    const int i = threadIdx.x;
    if (i >= nslabs || blockIdx.x != 0) return;
    double S[kSums] = {0.0, 0.0, 0.0, 0.0};
    for (int j = 0; j < nshares; j++)
        for (int k = 0; k < kSums; k++) S[k] += A.share[j][k];
    DevScalars s = *A.sc[i];
    if (s.status != LAT_OK) return;
    advance_scalars(M, s, S, advance != 0);
    s.ticket = 0u;
    *A.sc[i] = s;
}

// Equal-sized device regions copied in one launch (the halo planes of the slabs
// a process holds): blockIdx.y picks the region, the x blocks stride over its
// 16-byte words, four in flight per thread.
constexpr int kCopyChunk = 64;

struct CopyList {
    const uint4* src[kCopyChunk];
    uint4* dst[kCopyChunk];
};

__global__ void __launch_bounds__(256) copy_regions_kernel(CopyList L, size_t words)
{
    const uint4* __restrict__ s = L.src[blockIdx.y];
    uint4* __restrict__ d = L.dst[blockIdx.y];
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < words; i += 4 * stride) {
        const uint4 a = s[i], b = s[i + stride], c = s[i + 2 * stride], e = s[i + 3 * stride];
        d[i] = a;
        d[i + stride] = b;
        d[i + 2 * stride] = c;
        d[i + 3 * stride] = e;
    }
    for (; i < words; i += stride) d[i] = s[i];
}

int slab_sum_blocks(int n)
{
    const long long cols = (long long)n * n;
    return (int)std::max<long long>(1, std::min<long long>((cols + 255) / 256, 1024));
}

} // namespace

} // namespace lat

using namespace lat;

extern "C" {

lat_status lat_slab_create(const lat_params* params, int z0, int nzl, void* cuda_stream, void* const dev_bufs[8],
                           lat_handle** out)
{
    if (!out) return LAT_EINVAL;
    *out = nullptr;
    if (!params || !dev_bufs) return LAT_EINVAL;
    if (z0 < 0 || z0 >= params->n || nzl < 2 || nzl > params->n) return LAT_EINVAL;
    if (params->stencil == 27) return LAT_EUNSUPPORTED;   // the slab step is written for 7 points
    if (params->expansion == 2) return LAT_EUNSUPPORTED;  // and for eq. scale
    lat_handle* h = nullptr;
    LAT_TRY(lat_create_with_buffers(params, cuda_stream, dev_bufs, &h));
    h->slab = true;
    h->slab_z0 = z0;
    h->slab_nzl = nzl;
    h->nsites = (size_t)(nzl + 3) * params->n * params->n;
    h->dirty = false;
    MarchConfig cfg;
    if (!march_slab_config(params->n, (int)h->esize, nzl, &cfg) || (size_t)cfg.blocks * kSums > h->partials_cap ||
        (size_t)slab_sum_blocks(params->n) * kSums > h->partials_cap) {
        lat_destroy(h);
        return LAT_EUNSUPPORTED;
    }
    h->mcfg = cfg;
    h->variant = 2;
    h->ty = cfg.ty;
    h->zr = cfg.zr;
    drop_graph(h);
    *out = h;
    return LAT_OK;
}

lat_status lat_slab_sums(lat_handle* h, double* sums_dev)
{
    if (!h || !sums_dev) return LAT_EINVAL;
    if (!h->slab) return LAT_ESTATE;
    const int nb = slab_sum_blocks(h->M.n);
    if (h->prec == 32)
        slab_sums_kernel<float><<<nb, 256, 0, h->stream>>>(bufs_of<float>(h), h->M, h->sc, h->partials, h->slab_nzl,
                                                           sums_dev);
    else
        slab_sums_kernel<double><<<nb, 256, 0, h->stream>>>(bufs_of<double>(h), h->M, h->sc, h->partials,
                                                            h->slab_nzl, sums_dev);
    return cuda_status(cudaGetLastError());
}

lat_status lat_slab_step_range(lat_handle* h, int zfirst, int zcount, double* sums_dev)
{
    if (!h || !sums_dev) return LAT_EINVAL;
    if (!h->slab) return LAT_ESTATE;
    if (zfirst < 0 || zcount < 1 || zfirst + zcount > h->slab_nzl) return LAT_EINVAL;
    // the range's stored planes start at 1 + zfirst; the kernels read one plane
    // below it and two above, all within the slab's nzl + 3 stored planes
    const int n = h->M.n;
    MarchConfig cfg;
    cudaError_t e;
    if (slab_xw_config(n, (int)h->esize, zcount, &cfg) && (size_t)cfg.blocks * kSums <= h->partials_cap) {
        xw::SlabRun R = {};
        R.nranges = 1;
        R.nz = zcount;
        R.sums_out = sums_dev;
        R.rz[0] = 0;
        R.rn[0] = zcount;
        R.rzb[0] = 1 + zfirst;
        R.rslab[0] = 0;
        for (int i = 0; i < 8; i++) R.buf[0][i] = h->buf[i];
        e = h->prec == 32 ? launch_slab_xw<float>(R, h->M, h->sc, h->partials, cfg, h->stream)
                          : launch_slab_xw<double>(R, h->M, h->sc, h->partials, cfg, h->stream);
    } else {
        if (!march_slab_config(n, (int)h->esize, zcount, &cfg) || (size_t)cfg.blocks * kSums > h->partials_cap)
            return LAT_EUNSUPPORTED;
        cfg.zbase = 1 + zfirst;
        e = h->prec == 32 ? launch_step_march<float>(bufs_of<float>(h), h->M, h->sc, h->partials, cfg, h->stream,
                                                     sums_dev)
                          : launch_step_march<double>(bufs_of<double>(h), h->M, h->sc, h->partials, cfg, h->stream,
                                                      sums_dev);
    }
    return cuda_status(e);
}

lat_status lat_slab_step_ranges(lat_handle* const* slabs, int nslabs, const int32_t* ranges, int nranges,
                                double* sums_dev)
{
    if (!slabs || !ranges || !sums_dev || nslabs < 1 || nslabs > xw::kMaxLocalSlabs || nranges < 1 ||
        nranges > xw::kMaxSlabRanges)
        return LAT_EINVAL;
    lat_handle* h0 = slabs[0];
    for (int i = 0; i < nslabs; i++) {
        const lat_handle* h = slabs[i];
        if (!h) return LAT_EINVAL;
        if (!h->slab) return LAT_ESTATE;
        if (h->p.n != h0->p.n || h->prec != h0->prec || h->p.model != h0->p.model ||
            h->p.expansion != h0->p.expansion || h->p.dt != h0->p.dt || h->p.L != h0->p.L)
            return LAT_EINVAL;   // not slabs of one lattice
    }
    xw::SlabRun R = {};
    R.nranges = nranges;
    R.sums_out = sums_dev;
    int total = 0;
    for (int r = 0; r < nranges; r++) {
        const int s = ranges[3 * r], zfirst = ranges[3 * r + 1], zcount = ranges[3 * r + 2];
        if (s < 0 || s >= nslabs || zfirst < 0 || zcount < 1 || zfirst + zcount > slabs[s]->slab_nzl) return LAT_EINVAL;
        R.rz[r] = total;
        R.rn[r] = zcount;
        R.rzb[r] = 1 + zfirst;
        R.rslab[r] = s;
        total += zcount;
    }
    R.nz = total;
    for (int s = 0; s < nslabs; s++)
        for (int i = 0; i < 8; i++) R.buf[s][i] = slabs[s]->buf[i];
    MarchConfig cfg;
    if (!slab_xw_config(h0->M.n, (int)h0->esize, total, &cfg) || (size_t)cfg.blocks * kSums > h0->partials_cap)
        return LAT_EUNSUPPORTED;
    const cudaError_t e = h0->prec == 32 ? launch_slab_xw<float>(R, h0->M, h0->sc, h0->partials, cfg, h0->stream)
                                         : launch_slab_xw<double>(R, h0->M, h0->sc, h0->partials, cfg, h0->stream);
    return cuda_status(e);
}

lat_status lat_slab_step(lat_handle* h, double* sums_dev)
{
    if (!h || !sums_dev) return LAT_EINVAL;
    if (!h->slab) return LAT_ESTATE;
    return lat_slab_step_range(h, 0, h->slab_nzl, sums_dev);
}

lat_status lat_slab_advance(lat_handle* h, const double* sums_dev, int advance)
{
    if (!h || !sums_dev) return LAT_EINVAL;
    if (!h->slab) return LAT_ESTATE;
    slab_advance_kernel<<<1, 32, 0, h->stream>>>(h->M, h->sc, sums_dev, advance);
    return cuda_status(cudaGetLastError());
}

lat_status lat_slab_advance_local(lat_handle* const* slabs, int nslabs, const double* const* shares, int nshares,
                                  int advance)
{
    if (!slabs || !shares || nslabs < 1 || nslabs > kMaxLocalSlabs || nshares < 1 || nshares > kMaxLocalShares)
        return LAT_EINVAL;
    LocalAdvance A = {};
    for (int i = 0; i < nslabs; i++) {
        const lat_handle* h = slabs[i];
        if (!h) return LAT_EINVAL;
        if (!h->slab) return LAT_ESTATE;
        if (h->p.n != slabs[0]->p.n || h->prec != slabs[0]->prec || h->p.model != slabs[0]->p.model ||
            h->p.expansion != slabs[0]->p.expansion || h->p.dt != slabs[0]->p.dt || h->p.L != slabs[0]->p.L)
            return LAT_EINVAL;   // not slabs of one lattice
        A.sc[i] = h->sc;
    }
    for (int j = 0; j < nshares; j++) {
        if (!shares[j]) return LAT_EINVAL;
        A.share[j] = shares[j];
    }
    slab_advance_local_kernel<<<1, 64, 0, slabs[0]->stream>>>(slabs[0]->M, A, nslabs, nshares, advance);
    return cuda_status(cudaGetLastError());
}

lat_status lat_copy_regions(void* const* dst, const void* const* src, int count, uint64_t bytes, void* cuda_stream)
{
    if (!dst || !src || count < 0) return LAT_EINVAL;
    if (count == 0 || bytes == 0) return LAT_OK;
    if (bytes % 16 != 0) return LAT_EINVAL;
    for (int i = 0; i < count; i++)
        if (!dst[i] || !src[i] || ((uintptr_t)dst[i] | (uintptr_t)src[i]) % 16 != 0) return LAT_EINVAL;
    const size_t words = bytes / 16;
    const unsigned int bx = (unsigned int)std::min<size_t>((words + 1023) / 1024, 128);
    for (int c0 = 0; c0 < count; c0 += kCopyChunk) {
        const int nc = std::min(kCopyChunk, count - c0);
        CopyList L = {};
        for (int i = 0; i < nc; i++) {
            L.src[i] = (const uint4*)src[c0 + i];
            L.dst[i] = (uint4*)dst[c0 + i];
        }
        copy_regions_kernel<<<dim3(bx, (unsigned int)nc), 256, 0, (cudaStream_t)cuda_stream>>>(L, words);
        LAT_CUDA(cudaGetLastError());
    }
    return LAT_OK;
}

} // extern "C"
