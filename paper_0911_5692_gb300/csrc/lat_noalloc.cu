// lat_noalloc.cu -- lat_field_sums_static: the volume sums of a pair of field
// arrays, computed without allocating any device memory.
//
// Some callers cannot call cudaMalloc: a framework whose caching allocator has
// already reserved the device's memory, a service that must stay inside a fixed
// memory budget, or latency-sensitive code that cannot afford cudaMalloc's
// implicit device-wide synchronisation. For them this entry point runs the
// same per-block reduction as the sums pass of a lattice handle, but keeps its
// scratch (the per-block partial sums and the last-block counter) in one
// file-scope device array. Every GPU that loads the library holds that array
// (about 33 KB) until the process exits.
#include <algorithm>
#include <mutex>

#include "lat_common.cuh"

namespace lat {

namespace {

constexpr int kStaticBlocks = 1024;                   // most blocks one call uses
constexpr int kStaticThreads = 256;
constexpr size_t kTicketBytes = 256;                  // counter, padded to the array alignment
constexpr size_t kScratchBytes = kTicketBytes + (size_t)kStaticBlocks * kSums * sizeof(double);
constexpr int kMaxDevices = 64;

// The scratch: [last-block counter | per-block partials]. Shared by every call
// on a device; see the entry point for the rules that follow from that.
__device__ __align__(256) unsigned char g_sums_scratch[kScratchBytes];

// The sums of a handle's sums pass, in FP64 arithmetic: forward-difference
// |grad f|^2 of both fields (unscaled), f0^beta/beta and f0^2 f1^2/2,
// accumulated in FP64 per thread over (x, y) columns marched in z, then a
// fixed-order block and last-block reduction. The last block writes the volume
// averages and clears the counter.
template <typename T>
__global__ void __launch_bounds__(kStaticThreads) field_sums_static_kernel(const T* __restrict__ f0,
                                                                          const T* __restrict__ f1, int n,
                                                                          double inv_dx2, int beta, double* out,
                                                                          unsigned char* scratch)
{
    __shared__ double red[32 * kSums];
    __shared__ unsigned int is_last;
    unsigned int* ticket = reinterpret_cast<unsigned int*>(scratch);
    double* partials = reinterpret_cast<double*>(scratch + kTicketBytes);
    double acc[kSums] = {0.0, 0.0, 0.0, 0.0};
    const long long cols = (long long)n * n;
    for (long long col = (long long)blockIdx.x * blockDim.x + threadIdx.x; col < cols;
         col += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(col % n), y = (int)(col / n);
        const int xp = x == n - 1 ? 0 : x + 1, yp = y == n - 1 ? 0 : y + 1;
        for (int z = 0; z < n; z++) {
            const int zp = z == n - 1 ? 0 : z + 1;
            const size_t c = ((size_t)z * n + y) * n + x;
            const double a0 = (double)f0[c], a1 = (double)f1[c];
            const double e0 = (double)f0[((size_t)z * n + y) * n + xp] - a0;
            const double e1 = (double)f0[((size_t)z * n + yp) * n + x] - a0;
            const double e2 = (double)f0[((size_t)zp * n + y) * n + x] - a0;
            const double h0 = (double)f1[((size_t)z * n + y) * n + xp] - a1;
            const double h1 = (double)f1[((size_t)z * n + yp) * n + x] - a1;
            const double h2 = (double)f1[((size_t)zp * n + y) * n + x] - a1;
            acc[0] += e0 * e0 + e1 * e1 + e2 * e2;
            acc[1] += h0 * h0 + h1 * h1 + h2 * h2;
            const double sq = a0 * a0;
            acc[2] += beta == 4 ? 0.25 * sq * sq : 0.5 * sq;
            acc[3] += 0.5 * sq * a1 * a1;
        }
    }
    block_reduce(acc, red);
    if (threadIdx.x == 0) {
        for (int k = 0; k < kSums; k++) partials[(size_t)blockIdx.x * kSums + k] = acc[k];
        __threadfence();
        is_last = atomicAdd(ticket, 1u) == gridDim.x - 1u;
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double v[kSums] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
        for (int k = 0; k < kSums; k++) v[k] += __ldcg(partials + (size_t)b * kSums + k);
    block_reduce(v, red);
    if (threadIdx.x == 0) {
        const double inv_sites = 1.0 / ((double)n * n * n);
        out[0] = v[0] * inv_dx2 * inv_sites;
        out[1] = v[1] * inv_dx2 * inv_sites;
        out[2] = v[2] * inv_sites;
        out[3] = v[3] * inv_sites;
        *ticket = 0u;
    }
}

std::mutex g_setup_mutex;
unsigned char* g_scratch_addr[kMaxDevices];

// Device address of the scratch array on the current device, looked up (and the
// counter cleared) on the first call made on that device. The address is kept
// for the life of the process: a device reset (cudaDeviceReset) would leave it
// stale, so the entry point is not to be used across one.
cudaError_t scratch_for_current_device(unsigned char** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_sums_scratch);
        if (e != cudaSuccess) return e;
        e = cudaMemset(p, 0, kTicketBytes);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

} // namespace

} // namespace lat

extern "C" lat_status lat_field_sums_static(const void* f_phi, const void* f_chi, int n, int precision, int model,
                                            double L, double* out_dev, void* cuda_stream)
{
    using namespace lat;
    if (!f_phi || !f_chi || !out_dev) return LAT_EINVAL;
    if (precision != 32 && precision != 64) return LAT_EINVAL;
    if (model != LAT_MODEL_LPHI4 && model != LAT_MODEL_M2PHI2) return LAT_EINVAL;
    if (!(L > 0.0)) return LAT_EINVAL;
    if (n < 4) return LAT_EINVAL;
    // the lattice sides the library serves (lat_params.n): the range this entry
    // point is tested over; its scratch itself does not depend on n
    if (n > 1024) return LAT_EUNSUPPORTED;
    unsigned char* scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess) return LAT_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const long long cols = (long long)n * n;
    const int blocks = (int)std::min<long long>(kStaticBlocks, (cols + kStaticThreads - 1) / kStaticThreads);
    // the counter must start at zero; a completed call leaves it at zero, this
    // also covers a call that never finished
    if (cudaMemsetAsync(scratch, 0, sizeof(unsigned int), st) != cudaSuccess) return LAT_ECUDA;
    const double dx = L / n;
    const int beta = model == LAT_MODEL_LPHI4 ? 4 : 2;
    if (precision == 32)
        field_sums_static_kernel<float><<<blocks, kStaticThreads, 0, st>>>(
            static_cast<const float*>(f_phi), static_cast<const float*>(f_chi), n, 1.0 / (dx * dx), beta, out_dev,
            scratch);
    else
        field_sums_static_kernel<double><<<blocks, kStaticThreads, 0, st>>>(
            static_cast<const double*>(f_phi), static_cast<const double*>(f_chi), n, 1.0 / (dx * dx), beta, out_dev,
            scratch);
    return cudaGetLastError() == cudaSuccess ? LAT_OK : LAT_ECUDA;
}
