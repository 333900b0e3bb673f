// gt_kernels_mixed.cu -- mixed-precision transport kernels for the basic
// gas (isotropic levels, no attachment, uniform ionisation split), and the
// mixed-precision launch entry points, which pick the basic or the general
// instantiation (gt_kernels_mixed_phys.cu) from the uploaded gas.
#include "gt_kernels_mixed.inl"

namespace gt {

// the general instantiation lives in gt_kernels_mixed_phys.cu
extern template cudaError_t launch_batched_mixed_t<true>(const RunParams &, bool, int, int,
                                                         size_t, cudaStream_t);
extern template cudaError_t launch_plain_mixed_t<true>(const RunParams &, const PlainArgs &, bool,
                                                       int, size_t, cudaStream_t);
extern template cudaError_t configure_mixed_t<true>(size_t);

template cudaError_t launch_batched_mixed_t<false>(const RunParams &, bool, int, int, size_t,
                                                   cudaStream_t);
template cudaError_t launch_plain_mixed_t<false>(const RunParams &, const PlainArgs &, bool, int,
                                                 size_t, cudaStream_t);
template cudaError_t configure_mixed_t<false>(size_t);
template int occupancy_batched_mixed_t<false>(int, bool, int, size_t);

cudaError_t launch_batched_mixed(const RunParams &p, bool smem_table, int grid, int block,
                                 size_t smem, cudaStream_t s)
{
    return p.gas.any_special ? launch_batched_mixed_t<true>(p, smem_table, grid, block, smem, s)
                             : launch_batched_mixed_t<false>(p, smem_table, grid, block, smem, s);
}

cudaError_t launch_plain_mixed(const RunParams &p, const PlainArgs &a, bool smem_table, int block,
                               size_t smem, cudaStream_t s)
{
    return p.gas.any_special ? launch_plain_mixed_t<true>(p, a, smem_table, block, smem, s)
                             : launch_plain_mixed_t<false>(p, a, smem_table, block, smem, s);
}

cudaError_t configure_mixed(size_t max_smem)
{
    cudaError_t e = configure_mixed_t<false>(max_smem);
    if (e != cudaSuccess) return e;
    return configure_mixed_t<true>(max_smem);
}

int max_block_mixed() { return kMaxThreadsMixed; }

int occupancy_batched_mixed(int field_kind, bool smem_table, int block, size_t smem)
{
    return occupancy_batched_mixed_t<false>(field_kind, smem_table, block, smem);
}

}  // namespace gt
