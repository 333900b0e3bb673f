// gt_kernels_mixed.cu -- mixed-precision transport kernels for the basic
// gas (isotropic levels, no attachment, uniform ionisation split) and run
// (held field, post-flight endpoints), and the mixed-precision launch entry
// points, which pick the basic, PHYS or GEO variant from the gas and run.
#include "gt_kernels_mixed.inl"

namespace gt {

// the other variants live in gt_kernels_mixed_phys.cu and gt_kernels_mixed_geo.cu
#define GT_EXTERN_VARIANT(P, G)                                                                \
    extern template cudaError_t launch_batched_mixed_t<P, G>(const RunParams &, bool, int, int,   \
                                                             size_t, cudaStream_t);               \
    extern template cudaError_t launch_plain_mixed_t<P, G>(const RunParams &, const PlainArgs &, \
                                                           bool, int, size_t, cudaStream_t);      \
    extern template cudaError_t configure_mixed_t<P, G>(size_t);
GT_EXTERN_VARIANT(true, false)
GT_EXTERN_VARIANT(true, true)
#undef GT_EXTERN_VARIANT

template cudaError_t launch_batched_mixed_t<false, false>(const RunParams &, bool, int, int,
                                                          size_t, cudaStream_t);
template cudaError_t launch_plain_mixed_t<false, false>(const RunParams &, const PlainArgs &,
                                                        bool, int, size_t, cudaStream_t);
template cudaError_t configure_mixed_t<false, false>(size_t);
template int occupancy_batched_mixed_t<false, false>(int, bool, int, size_t);

// Variants: the basic gas; gases with anisotropy, attachment or a sharing
// law (PHYS); runs with sub-steps, exact crossings or induced signals (GEO,
// with PHYS).
static bool geo(const RunParams &p) { return p.substeps > 1 || p.crossing || p.signal_bins; }
static bool phys(const RunParams &p) { return p.gas.any_special != 0; }

cudaError_t launch_batched_mixed(const RunParams &p, bool smem_table, int grid, int block,
                                 size_t smem, cudaStream_t s)
{
    if (geo(p)) return launch_batched_mixed_t<true, true>(p, smem_table, grid, block, smem, s);
    if (phys(p)) return launch_batched_mixed_t<true, false>(p, smem_table, grid, block, smem, s);
    return launch_batched_mixed_t<false, false>(p, smem_table, grid, block, smem, s);
}

cudaError_t launch_plain_mixed(const RunParams &p, const PlainArgs &a, bool smem_table, int block,
                               size_t smem, cudaStream_t s)
{
    if (geo(p)) return launch_plain_mixed_t<true, true>(p, a, smem_table, block, smem, s);
    if (phys(p)) return launch_plain_mixed_t<true, false>(p, a, smem_table, block, smem, s);
    return launch_plain_mixed_t<false, false>(p, a, smem_table, block, smem, s);
}

cudaError_t configure_mixed(size_t max_smem)
{
    cudaError_t e = configure_mixed_t<false, false>(max_smem);
    if (e != cudaSuccess) return e;
    if ((e = configure_mixed_t<true, false>(max_smem)) != cudaSuccess) return e;
    return configure_mixed_t<true, true>(max_smem);
}

int max_block_mixed() { return kMaxThreadsMixed; }

int occupancy_batched_mixed(int field_kind, bool smem_table, int block, size_t smem)
{
    return occupancy_batched_mixed_t<false, false>(field_kind, smem_table, block, smem);
}

}  // namespace gt
