// gt_kernels_mixed_geo_gtab.cu -- the sub-step, crossing and signal variant's
// kernels that read the FP32 table from global memory (tables too large for
// shared memory); split from gt_kernels_mixed_geo.cu so that the two compile
// in parallel.
#include "gt_kernels_mixed.inl"

namespace gt {

template cudaError_t launch_batched_mixed_tab<false, true, true>(const RunParams &, int, int, size_t,
                                                                 cudaStream_t);
template cudaError_t launch_plain_mixed_tab<false, true, true>(const RunParams &,
                                                               const PlainArgs &, int, size_t,
                                                               cudaStream_t);
template cudaError_t configure_mixed_tab<false, true, true>(size_t);
template int occupancy_batched_mixed_tab<false, true, true>(int, int, size_t);

}  // namespace gt
