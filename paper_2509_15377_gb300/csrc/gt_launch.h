// gt_launch.h -- host-side launchers shared by the runtime (gt_api.cu) and
// the kernel translation units.  Internal to the library.
#pragma once

#include <cuda_runtime.h>

#include "gt_device.cuh"

struct gt_ctx;

namespace gt {

// Device index of a context (gt_api.cu), -1 for NULL.
int context_device(const gt_ctx *ctx);

// Static shared memory of the transport kernels stays below this; the
// dynamic part (tallies and table) may use the rest of a CTA's opt-in size.
constexpr size_t kStaticSmemReserve = 4096;

// Let a kernel use all the dynamic shared memory a CTA may have beyond the
// kernel's own static shared memory.
template <typename F>
inline cudaError_t allow_dynamic_smem(F *kernel, size_t optin)
{
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, kernel);
    if (e != cudaSuccess) return e;
    const size_t dyn = optin > a.sharedSizeBytes ? optin - a.sharedSizeBytes : 0;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
}

struct SeedArgs {
    const double *x, *y, *z, *t, *e, *dx, *dy, *dz;
    const int32_t *aval;
    const uint64_t *uid;
    long long n;
    int unfilled_slot;  // fault injection: reserve one slot that is never filled
};

struct PlainArgs {
    Stack cur, fresh, next;
    long long n_active;
    int parity;
    int aval;
};

// Per-precision transport launchers (gt_kernels_fp64.cu / gt_kernels_mixed.cu).
// `smem_table` selects the shared-memory copy of the FP32 table.
cudaError_t launch_batched_fp64(const RunParams &p, int grid, int block, size_t smem,
                                cudaStream_t s);
cudaError_t launch_batched_mixed(const RunParams &p, bool smem_table, int grid, int block,
                                 size_t smem, cudaStream_t s);
cudaError_t launch_plain_fp64(const RunParams &p, const PlainArgs &a, int block, size_t smem,
                              cudaStream_t s);
cudaError_t launch_plain_mixed(const RunParams &p, const PlainArgs &a, bool smem_table, int block,
                               size_t smem, cudaStream_t s);
// The mixed launchers above dispatch on the gas and the run: the general
// collision (PHYS) and the sub-steps / crossings (GEO) are separate builds
// of the kernels (gt_kernels_mixed.inl).
template <bool PHYS, bool GEO>
cudaError_t launch_batched_mixed_t(const RunParams &p, bool smem_table, int grid, int block,
                                   size_t smem, cudaStream_t s);
template <bool PHYS, bool GEO>
cudaError_t launch_plain_mixed_t(const RunParams &p, const PlainArgs &a, bool smem_table,
                                 int block, size_t smem, cudaStream_t s);
template <bool PHYS, bool GEO>
cudaError_t configure_mixed_t(size_t max_smem);
template <bool PHYS, bool GEO>
int occupancy_batched_mixed_t(int field_kind, bool smem_table, int block, size_t smem);
// Raise the dynamic shared-memory limit of every transport instantiation.
cudaError_t configure_fp64(size_t max_smem);
cudaError_t configure_mixed(size_t max_smem);
int max_block_fp64();
int max_block_mixed();
// Resident CTAs per SM of the batched kernel for this launch shape.
int occupancy_batched_fp64(int field_kind, int block, size_t smem);
int occupancy_batched_mixed(int field_kind, bool smem_table, int block, size_t smem);

// gt_common.cu
cudaError_t launch_seed(const RunParams &p, const SeedArgs &a, cudaStream_t s);
cudaError_t launch_plain_init(const RunParams &p, const Stack &st, const long long *order,
                              long long first, long long count, cudaStream_t s);
cudaError_t launch_plain_compact(const RunParams &p, const PlainArgs &a, cudaStream_t s);
cudaError_t launch_count_electrons(const RunParams &p, int sms, cudaStream_t s);
// Largest |E| over the nodes of a device grid map (synchronous; setup only).
cudaError_t grid_emax(const float4 *grid, long long n, int sms, double *emax);
cudaError_t launch_observables(const RunParams &p, long long n_endpoints, int n_avalanches,
                               const int32_t *n_prim, int collect_status, int drift_status,
                               double gap, unsigned long long *scratch_counts,
                               double *scratch_partials, int n_blocks, double *obs,
                               cudaStream_t s);

}  // namespace gt
