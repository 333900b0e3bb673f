// gt_kernels_mixed_geo.cu -- mixed-precision transport kernels for runs with flights in sub-steps or exact boundary crossings (any gas).
#include "gt_kernels_mixed.inl"

namespace gt {

template cudaError_t launch_batched_mixed_t<true, true>(const RunParams &, bool, int, int, size_t,
                                                       cudaStream_t);
template cudaError_t launch_plain_mixed_t<true, true>(const RunParams &, const PlainArgs &, bool,
                                                     int, size_t, cudaStream_t);
template cudaError_t configure_mixed_t<true, true>(size_t);
template int occupancy_batched_mixed_t<true, true>(int, bool, int, size_t);

}  // namespace gt
