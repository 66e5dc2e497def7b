// lat_grid.h -- launch shape of the column-marching passes (the sums after an
// upload, the L = 1/H form's pass, the per-site energy field): one resident
// wave of blocks, each thread marching whole z runs of one column.
#pragma once

#include <cuda_runtime.h>

namespace lat {

// Runs per column for `cols` columns of n planes over `threads` threads, where
// a run of k planes costs k + startup plane-times (the planes loaded before its
// first one): the count in [1, n/4] that minimises (runs per thread) x (n/runs +
// startup), the time of the busiest thread.
inline int balanced_zruns(long long cols, int n, long long threads, double startup)
{
    int best_c = 1;
    double best = 0.0;
    for (int c = 1; c <= (n / 4 > 1 ? n / 4 : 1); c++) {
        const long long per_thread = (cols * c + threads - 1) / threads;
        const double cost = (double)per_thread * ((double)n / c + startup);
        if (c == 1 || cost < best) {
            best = cost;
            best_c = c;
        }
    }
    return best_c;
}

// Resident blocks per SM of `kernel` at `threads` threads (cached by the
// caller), times the SM count of the current device; 0 on error.
inline int resident_wave(const void* kernel, int threads, int* occ_cache)
{
    if (*occ_cache == 0) {
        int o = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, kernel, threads, 0) != cudaSuccess || o < 1) o = 1;
        *occ_cache = o;
    }
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return *occ_cache * sms;
}

} // namespace lat
