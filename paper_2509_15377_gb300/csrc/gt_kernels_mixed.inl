// gt_kernels_mixed.inl -- mixed-precision instantiations of the transport
// kernels, as templates on PHYS (the general collision with anisotropy,
// attachment and a sharing law, or the basic gas's collision without their
// code) and GEO (flights in sub-steps and exact boundary crossings, or not).
// Included by gt_kernels_mixed.cu (basic), gt_kernels_mixed_phys.cu (PHYS)
// and gt_kernels_mixed_geo.cu (PHYS and GEO), which instantiate one variant
// each so that they compile in parallel.  The FP32 cumulative table is staged in
// shared memory when it fits next to the per-thread tallies (else read
// through the read-only path).
#pragma once

#include "gt_kernels.cuh"
#include "gt_launch.h"

namespace gt {

// The batched kernel is built for four launch bounds: more resident warps
// per SM against fewer registers per thread (the FP32 table in shared
// memory limits an SM to one CTA).
constexpr int kMaxThreadsMixed = 1024;
constexpr int kPlainThreadsMixed = 512;

// The run the step has a build of its own for (kRoundCommon): one flight per
// round, the banded majorant with band bounds rising with energy, an
// elastic level 0, no magnetic field, the field held over each flight.
static bool common_run(const RunParams &p)
{
    return p.flights_per_phase == 1 && p.majorant == GT_MAJORANT_BANDED &&
           p.gas.bands_monotone && p.gas.level0_elastic && !p.field.has_b &&
           p.field_emax_f == 0.0f;
}

// The common run with exact crossings and neither sub-steps nor signals
// (kRoundCrossing, the plate field in the GEO variant).
static bool crossing_only_run(const RunParams &p)
{
    return common_run(p) && p.crossing && p.substeps <= 1 && !p.signal_bins;
}

// The common run with induced signals and neither sub-steps nor crossings
// (kRoundSignal, the plate field in the GEO variant).
static bool signal_only_run(const RunParams &p)
{
    return common_run(p) && p.signal_bins > 0 && !p.crossing && p.substeps <= 1;
}

template <int FK, bool TAB, int MAXT, bool PHYS, bool GEO>
static cudaError_t batched_t(const RunParams &p, int grid, int block, size_t smem, cudaStream_t s)
{
    if constexpr (GEO && FK == GT_FIELD_PLATE) {
        if (crossing_only_run(p)) {
            k_batched<MixedElectron, FK, TAB, MAXT, kRoundCrossing, PHYS, GEO>
                <<<grid, block, smem, s>>>(p);
            return cudaGetLastError();
        }
        if (signal_only_run(p)) {
            k_batched<MixedElectron, FK, TAB, MAXT, kRoundSignal, PHYS, GEO>
                <<<grid, block, smem, s>>>(p);
            return cudaGetLastError();
        }
    }
    // built for every field in the basic variant, for the plate field in the others
    if constexpr ((!PHYS && !GEO) || FK == GT_FIELD_PLATE) {
        if (common_run(p)) {
            k_batched<MixedElectron, FK, TAB, MAXT, kRoundCommon, PHYS, GEO>
                <<<grid, block, smem, s>>>(p);
            return cudaGetLastError();
        }
    }
    if (p.flights_per_phase == 1)
        k_batched<MixedElectron, FK, TAB, MAXT, kRoundOne, PHYS, GEO><<<grid, block, smem, s>>>(p);
    else
        k_batched<MixedElectron, FK, TAB, MAXT, kRoundAny, PHYS, GEO><<<grid, block, smem, s>>>(p);
    return cudaGetLastError();
}

template <int FK, bool TAB, bool PHYS, bool GEO>
static cudaError_t batched(const RunParams &p, int grid, int block, size_t smem, cudaStream_t s)
{
    if (block <= 512) return batched_t<FK, TAB, 512, PHYS, GEO>(p, grid, block, smem, s);
    if (block <= 768) return batched_t<FK, TAB, 768, PHYS, GEO>(p, grid, block, smem, s);
    if (block <= 896) return batched_t<FK, TAB, 896, PHYS, GEO>(p, grid, block, smem, s);
    return batched_t<FK, TAB, 1024, PHYS, GEO>(p, grid, block, smem, s);
}

template <int FK, bool TAB, bool PHYS, bool GEO>
static cudaError_t plain(const RunParams &p, const PlainArgs &a, int block, size_t smem,
                         cudaStream_t s)
{
    const long long n = a.n_active;
    if (n <= 0) return cudaSuccess;
    k_plain_transport<MixedElectron, FK, TAB, kPlainThreadsMixed, PHYS, GEO>
        <<<(unsigned)((n + block - 1) / block), block, smem, s>>>(p, a.cur, n, a.fresh, a.parity,
                                                                  a.aval);
    return cudaGetLastError();
}

template <bool TAB, bool PHYS, bool GEO>
static cudaError_t batched_fk(const RunParams &p, int grid, int block, size_t smem, cudaStream_t s)
{
    switch (p.field.kind) {
    case GT_FIELD_UNIFORM: return batched<GT_FIELD_UNIFORM, TAB, PHYS, GEO>(p, grid, block, smem, s);
    case GT_FIELD_PLATE: return batched<GT_FIELD_PLATE, TAB, PHYS, GEO>(p, grid, block, smem, s);
    case GT_FIELD_COAX: return batched<GT_FIELD_COAX, TAB, PHYS, GEO>(p, grid, block, smem, s);
    case GT_FIELD_MESH: return batched<GT_FIELD_MESH, TAB, PHYS, GEO>(p, grid, block, smem, s);
    default: return batched<GT_FIELD_GRID, TAB, PHYS, GEO>(p, grid, block, smem, s);
    }
}

template <bool TAB, bool PHYS, bool GEO>
static cudaError_t plain_fk(const RunParams &p, const PlainArgs &a, int block, size_t smem,
                            cudaStream_t s)
{
    switch (p.field.kind) {
    case GT_FIELD_UNIFORM: return plain<GT_FIELD_UNIFORM, TAB, PHYS, GEO>(p, a, block, smem, s);
    case GT_FIELD_PLATE: return plain<GT_FIELD_PLATE, TAB, PHYS, GEO>(p, a, block, smem, s);
    case GT_FIELD_COAX: return plain<GT_FIELD_COAX, TAB, PHYS, GEO>(p, a, block, smem, s);
    case GT_FIELD_MESH: return plain<GT_FIELD_MESH, TAB, PHYS, GEO>(p, a, block, smem, s);
    default: return plain<GT_FIELD_GRID, TAB, PHYS, GEO>(p, a, block, smem, s);
    }
}

// Entry points per table placement (TAB: the FP32 table in shared memory),
// so that a variant's kernels can be split over two translation units by
// TAB and compiled in parallel (the GEO variant is).
template <bool TAB, bool PHYS, bool GEO>
cudaError_t launch_batched_mixed_tab(const RunParams &p, int grid, int block, size_t smem,
                                     cudaStream_t s)
{
    return batched_fk<TAB, PHYS, GEO>(p, grid, block, smem, s);
}

template <bool TAB, bool PHYS, bool GEO>
cudaError_t launch_plain_mixed_tab(const RunParams &p, const PlainArgs &a, int block, size_t smem,
                                   cudaStream_t s)
{
    return plain_fk<TAB, PHYS, GEO>(p, a, block, smem, s);
}

template <bool PHYS, bool GEO>
cudaError_t launch_batched_mixed_t(const RunParams &p, bool smem_table, int grid, int block,
                                   size_t smem, cudaStream_t s)
{
    return smem_table ? launch_batched_mixed_tab<true, PHYS, GEO>(p, grid, block, smem, s)
                      : launch_batched_mixed_tab<false, PHYS, GEO>(p, grid, block, smem, s);
}

template <bool PHYS, bool GEO>
cudaError_t launch_plain_mixed_t(const RunParams &p, const PlainArgs &a, bool smem_table,
                                 int block, size_t smem, cudaStream_t s)
{
    return smem_table ? launch_plain_mixed_tab<true, PHYS, GEO>(p, a, block, smem, s)
                      : launch_plain_mixed_tab<false, PHYS, GEO>(p, a, block, smem, s);
}

template <int FK, bool TAB, int MP, bool PHYS, bool GEO>
static cudaError_t configure_mp(size_t max_smem)
{
    cudaError_t e;
    if ((e = allow_dynamic_smem(k_batched<MixedElectron, FK, TAB, 512, MP, PHYS, GEO>, max_smem)) !=
        cudaSuccess)
        return e;
    if ((e = allow_dynamic_smem(k_batched<MixedElectron, FK, TAB, 768, MP, PHYS, GEO>, max_smem)) !=
        cudaSuccess)
        return e;
    if ((e = allow_dynamic_smem(k_batched<MixedElectron, FK, TAB, 896, MP, PHYS, GEO>, max_smem)) !=
        cudaSuccess)
        return e;
    return allow_dynamic_smem(k_batched<MixedElectron, FK, TAB, 1024, MP, PHYS, GEO>, max_smem);
}

template <int FK, bool TAB, bool PHYS, bool GEO>
static cudaError_t configure_one(size_t max_smem)
{
    cudaError_t e;
    if ((e = configure_mp<FK, TAB, kRoundAny, PHYS, GEO>(max_smem)) != cudaSuccess) return e;
    if ((e = configure_mp<FK, TAB, kRoundOne, PHYS, GEO>(max_smem)) != cudaSuccess) return e;
    if constexpr ((!PHYS && !GEO) || FK == GT_FIELD_PLATE) {
        if ((e = configure_mp<FK, TAB, kRoundCommon, PHYS, GEO>(max_smem)) != cudaSuccess) return e;
    }
    if constexpr (GEO && FK == GT_FIELD_PLATE) {
        if ((e = configure_mp<FK, TAB, kRoundCrossing, PHYS, GEO>(max_smem)) != cudaSuccess) return e;
        if ((e = configure_mp<FK, TAB, kRoundSignal, PHYS, GEO>(max_smem)) != cudaSuccess) return e;
    }
    return allow_dynamic_smem(k_plain_transport<MixedElectron, FK, TAB, kPlainThreadsMixed, PHYS, GEO>,
                              max_smem);
}

template <bool TAB, bool PHYS, bool GEO>
static cudaError_t configure_tab(size_t max_smem)
{
    cudaError_t e;
    if ((e = configure_one<GT_FIELD_UNIFORM, TAB, PHYS, GEO>(max_smem)) != cudaSuccess) return e;
    if ((e = configure_one<GT_FIELD_PLATE, TAB, PHYS, GEO>(max_smem)) != cudaSuccess) return e;
    if ((e = configure_one<GT_FIELD_COAX, TAB, PHYS, GEO>(max_smem)) != cudaSuccess) return e;
    if ((e = configure_one<GT_FIELD_MESH, TAB, PHYS, GEO>(max_smem)) != cudaSuccess) return e;
    return configure_one<GT_FIELD_GRID, TAB, PHYS, GEO>(max_smem);
}

template <bool TAB, bool PHYS, bool GEO>
cudaError_t configure_mixed_tab(size_t max_smem)
{
    return configure_tab<TAB, PHYS, GEO>(max_smem);
}

template <bool PHYS, bool GEO>
cudaError_t configure_mixed_t(size_t max_smem)
{
    cudaError_t e = configure_mixed_tab<true, PHYS, GEO>(max_smem);
    if (e != cudaSuccess) return e;
    return configure_mixed_tab<false, PHYS, GEO>(max_smem);
}

template <int FK, bool TAB, bool PHYS, bool GEO>
static int occ(int block, size_t smem)
{
    int n = 0;
    cudaError_t e;
    if (block <= 512)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &n, k_batched<MixedElectron, FK, TAB, 512, kRoundAny, PHYS, GEO>, block, smem);
    else if (block <= 768)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &n, k_batched<MixedElectron, FK, TAB, 768, kRoundAny, PHYS, GEO>, block, smem);
    else if (block <= 896)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &n, k_batched<MixedElectron, FK, TAB, 896, kRoundAny, PHYS, GEO>, block, smem);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &n, k_batched<MixedElectron, FK, TAB, 1024, kRoundAny, PHYS, GEO>, block, smem);
    return e == cudaSuccess ? n : 0;
}

template <bool TAB, bool PHYS, bool GEO>
static int occ_fk(int field_kind, int block, size_t smem)
{
    switch (field_kind) {
    case GT_FIELD_UNIFORM: return occ<GT_FIELD_UNIFORM, TAB, PHYS, GEO>(block, smem);
    case GT_FIELD_PLATE: return occ<GT_FIELD_PLATE, TAB, PHYS, GEO>(block, smem);
    case GT_FIELD_COAX: return occ<GT_FIELD_COAX, TAB, PHYS, GEO>(block, smem);
    case GT_FIELD_MESH: return occ<GT_FIELD_MESH, TAB, PHYS, GEO>(block, smem);
    default: return occ<GT_FIELD_GRID, TAB, PHYS, GEO>(block, smem);
    }
}

template <bool TAB, bool PHYS, bool GEO>
int occupancy_batched_mixed_tab(int field_kind, int block, size_t smem)
{
    return occ_fk<TAB, PHYS, GEO>(field_kind, block, smem);
}

template <bool PHYS, bool GEO>
int occupancy_batched_mixed_t(int field_kind, bool smem_table, int block, size_t smem)
{
    return smem_table ? occupancy_batched_mixed_tab<true, PHYS, GEO>(field_kind, block, smem)
                      : occupancy_batched_mixed_tab<false, PHYS, GEO>(field_kind, block, smem);
}

}  // namespace gt
