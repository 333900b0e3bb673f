// gt_kernels_fp64.cu -- FP64 instantiations of the transport kernels.  The
// FP64 table is read through the read-only data path (it is twice the size
// of the FP32 one and the FP64 pipe, not the table, bounds this precision).
#include "gt_kernels.cuh"
#include "gt_launch.h"

namespace gt {

constexpr int kMaxThreads64 = 512;

template <int FK>
static cudaError_t batched(const RunParams &p, int grid, int block, size_t smem, cudaStream_t s)
{
    k_batched<Fp64Electron, FK, false, kMaxThreads64><<<grid, block, smem, s>>>(p);
    return cudaGetLastError();
}

template <int FK>
static cudaError_t plain(const RunParams &p, const PlainArgs &a, int block, size_t smem,
                         cudaStream_t s)
{
    const long long n = a.n_active;
    if (n <= 0) return cudaSuccess;
    k_plain_transport<Fp64Electron, FK, false, kMaxThreads64>
        <<<(unsigned)((n + block - 1) / block), block, smem, s>>>(p, a.cur, n, a.fresh, a.parity,
                                                                  a.aval);
    return cudaGetLastError();
}

cudaError_t launch_batched_fp64(const RunParams &p, int grid, int block, size_t smem,
                                cudaStream_t s)
{
    switch (p.field.kind) {
    case GT_FIELD_UNIFORM: return batched<GT_FIELD_UNIFORM>(p, grid, block, smem, s);
    case GT_FIELD_PLATE: return batched<GT_FIELD_PLATE>(p, grid, block, smem, s);
    case GT_FIELD_COAX: return batched<GT_FIELD_COAX>(p, grid, block, smem, s);
    case GT_FIELD_MESH: return batched<GT_FIELD_MESH>(p, grid, block, smem, s);
    default: return batched<GT_FIELD_GRID>(p, grid, block, smem, s);
    }
}

cudaError_t launch_plain_fp64(const RunParams &p, const PlainArgs &a, int block, size_t smem,
                              cudaStream_t s)
{
    switch (p.field.kind) {
    case GT_FIELD_UNIFORM: return plain<GT_FIELD_UNIFORM>(p, a, block, smem, s);
    case GT_FIELD_PLATE: return plain<GT_FIELD_PLATE>(p, a, block, smem, s);
    case GT_FIELD_COAX: return plain<GT_FIELD_COAX>(p, a, block, smem, s);
    case GT_FIELD_MESH: return plain<GT_FIELD_MESH>(p, a, block, smem, s);
    default: return plain<GT_FIELD_GRID>(p, a, block, smem, s);
    }
}

template <int FK>
static cudaError_t configure_one(size_t max_smem)
{
    cudaError_t e = allow_dynamic_smem(k_batched<Fp64Electron, FK, false, kMaxThreads64>, max_smem);
    if (e != cudaSuccess) return e;
    return allow_dynamic_smem(k_plain_transport<Fp64Electron, FK, false, kMaxThreads64>, max_smem);
}

cudaError_t configure_fp64(size_t max_smem)
{
    cudaError_t e;
    if ((e = configure_one<GT_FIELD_UNIFORM>(max_smem)) != cudaSuccess) return e;
    if ((e = configure_one<GT_FIELD_PLATE>(max_smem)) != cudaSuccess) return e;
    if ((e = configure_one<GT_FIELD_COAX>(max_smem)) != cudaSuccess) return e;
    if ((e = configure_one<GT_FIELD_MESH>(max_smem)) != cudaSuccess) return e;
    return configure_one<GT_FIELD_GRID>(max_smem);
}

int max_block_fp64() { return kMaxThreads64; }

template <int FK>
static int occ(int block, size_t smem)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &n, k_batched<Fp64Electron, FK, false, kMaxThreads64>, block, smem) != cudaSuccess)
        return 0;
    return n;
}

int occupancy_batched_fp64(int field_kind, int block, size_t smem)
{
    switch (field_kind) {
    case GT_FIELD_UNIFORM: return occ<GT_FIELD_UNIFORM>(block, smem);
    case GT_FIELD_PLATE: return occ<GT_FIELD_PLATE>(block, smem);
    case GT_FIELD_COAX: return occ<GT_FIELD_COAX>(block, smem);
    case GT_FIELD_MESH: return occ<GT_FIELD_MESH>(block, smem);
    default: return occ<GT_FIELD_GRID>(block, smem);
    }
}

}  // namespace gt
