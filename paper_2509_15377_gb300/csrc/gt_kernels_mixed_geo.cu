// gt_kernels_mixed_geo.cu -- mixed-precision transport kernels for runs with
// flights in sub-steps, exact boundary crossings or induced signals (any
// gas): the builds with the FP32 table in shared memory, and the variant's
// entry points.  The builds that read the table from global memory are in
// gt_kernels_mixed_geo_gtab.cu, compiled in parallel.
#include "gt_kernels_mixed.inl"

namespace gt {

extern template cudaError_t launch_batched_mixed_tab<false, true, true>(const RunParams &, int, int,
                                                                        size_t, cudaStream_t);
extern template cudaError_t launch_plain_mixed_tab<false, true, true>(const RunParams &,
                                                                      const PlainArgs &, int,
                                                                      size_t, cudaStream_t);
extern template cudaError_t configure_mixed_tab<false, true, true>(size_t);
extern template int occupancy_batched_mixed_tab<false, true, true>(int, int, size_t);

template cudaError_t launch_batched_mixed_t<true, true>(const RunParams &, bool, int, int, size_t,
                                                       cudaStream_t);
template cudaError_t launch_plain_mixed_t<true, true>(const RunParams &, const PlainArgs &, bool,
                                                     int, size_t, cudaStream_t);
template cudaError_t configure_mixed_t<true, true>(size_t);
template int occupancy_batched_mixed_t<true, true>(int, bool, int, size_t);

}  // namespace gt
