// lat_split.cu -- the arrays of split storage (lat_params.split): shifting a
// stored array by a constant when the homogeneous inflaton mode moves or whole
// fields are exchanged, and the volume means that lat_recenter moves into the
// homogeneous mode. Off the step path.
#include "lat_kernels.h"

namespace lat {

namespace {

// a[i] <- a[i] + delta, the sum formed in FP64 and rounded once
template <typename T>
__global__ void shift_kernel(T* a, size_t count, double delta)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        a[i] = (T)((double)a[i] + delta);
}

// Per-block FP64 sums of two arrays: partials[2 b], partials[2 b + 1].
template <typename T>
__global__ void __launch_bounds__(256) sum2_kernel(const T* a, const T* b, size_t count, double* partials)
{
    __shared__ double red[8][2];
    double sa = 0.0, sb = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        sa += (double)a[i];
        sb += (double)b[i];
    }
    for (int o = 16; o > 0; o >>= 1) {
        sa += __shfl_down_sync(0xffffffffu, sa, o);
        sb += __shfl_down_sync(0xffffffffu, sb, o);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        red[warp][0] = sa;
        red[warp][1] = sb;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += red[w][threadIdx.x];
        partials[2 * (size_t)blockIdx.x + threadIdx.x] = s;
    }
}

int grid_for(size_t count)
{
    const size_t blocks = (count + 255) / 256;
    return (int)(blocks < (size_t)kSum2Blocks ? blocks : (size_t)kSum2Blocks);
}

} // namespace

template <typename T>
cudaError_t launch_shift(T* a, size_t count, double delta, cudaStream_t st)
{
    if (count == 0 || delta == 0.0) return cudaSuccess;
    shift_kernel<T><<<grid_for(count), 256, 0, st>>>(a, count, delta);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sum2(const T* a, const T* b, size_t count, double* partials, int* blocks, cudaStream_t st)
{
    *blocks = grid_for(count);
    sum2_kernel<T><<<*blocks, 256, 0, st>>>(a, b, count, partials);
    return cudaGetLastError();
}

template cudaError_t launch_shift<float>(float*, size_t, double, cudaStream_t);
template cudaError_t launch_shift<double>(double*, size_t, double, cudaStream_t);
template cudaError_t launch_sum2<float>(const float*, const float*, size_t, double*, int*, cudaStream_t);
template cudaError_t launch_sum2<double>(const double*, const double*, size_t, double*, int*, cudaStream_t);

} // namespace lat
