// lat_step_tma.cu -- TMA plane-ring fused step (placeholder until the kernel lands).
#include "lat_kernels.h"

namespace lat {

bool tma_config(int, int, int, int, TmaConfig*) { return false; }

template <typename T>
cudaError_t launch_step_tma(const Bufs<T>&, const Model&, DevScalars*, double*, const TmaConfig&, const void*,
                            cudaStream_t)
{
    return cudaErrorNotSupported;
}

cudaError_t tma_encode_maps(const void* const*, int, int, void*) { return cudaErrorNotSupported; }

template cudaError_t launch_step_tma<float>(const Bufs<float>&, const Model&, DevScalars*, double*,
                                            const TmaConfig&, const void*, cudaStream_t);
template cudaError_t launch_step_tma<double>(const Bufs<double>&, const Model&, DevScalars*, double*,
                                             const TmaConfig&, const void*, cudaStream_t);

} // namespace lat
