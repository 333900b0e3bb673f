// gt_kernels_mixed_phys.cu -- mixed-precision transport kernels for the general gas (anisotropic scattering, attachment, a sharing law).
#include "gt_kernels_mixed.inl"

namespace gt {

template cudaError_t launch_batched_mixed_t<true, false>(const RunParams &, bool, int, int, size_t,
                                                       cudaStream_t);
template cudaError_t launch_plain_mixed_t<true, false>(const RunParams &, const PlainArgs &, bool,
                                                     int, size_t, cudaStream_t);
template cudaError_t configure_mixed_t<true, false>(size_t);
template int occupancy_batched_mixed_t<true, false>(int, bool, int, size_t);

}  // namespace gt
