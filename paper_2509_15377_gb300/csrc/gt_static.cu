// gt_static.cu -- avalanche_run_static: the batched run with its scratch
// memory in a fixed, file-scope device array instead of a caller-provided
// work space, so that the call allocates nothing.
//
// Who needs it: callers that cannot call cudaMalloc at the point where they
// run avalanches, e.g. code inside a framework whose memory manager owns the
// device memory, or a loop that must not pay the implicit device
// synchronisation an allocation or free can cause.  Such a caller still
// provides the inputs (device primaries) and the outputs (endpoint arrays,
// per-avalanche counts and tallies); only the scratch comes from here.
//
// The array is part of the library's device image: every GPU that loads the
// library holds it (GT_STATIC_SCRATCH_BYTES) until the process exits.
#include <mutex>

#include "gt_avalanche.h"
#include "gt_device.cuh"
#include "gt_launch.h"

namespace {

// Layout of the batched run's work space for GT_STATIC_MAX_ELECTRONS slots
// and GT_STATIC_MAX_AVALANCHES avalanches with device-resident primaries:
// header, ready flags (u32), birth velocity (3 x f64), birth element (i32),
// created counters (u64), every region rounded up to 256 bytes.
constexpr size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kStaticBytes =
    round256(sizeof(gt::Header)) + round256(sizeof(uint32_t) * GT_STATIC_MAX_ELECTRONS) +
    3 * round256(sizeof(double) * GT_STATIC_MAX_ELECTRONS) +
    round256(sizeof(int32_t) * GT_STATIC_MAX_ELECTRONS) +
    round256(sizeof(unsigned long long) * GT_STATIC_MAX_AVALANCHES) + 256;
static_assert(kStaticBytes == GT_STATIC_SCRATCH_BYTES, "header constant out of date");

// The scratch itself.  In host code this name is only a stand-in for the
// symbol: its device address is obtained per device with
// cudaGetSymbolAddress and passed to the kernels.
static __device__ __align__(256) unsigned char g_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_lock;
void *g_addr[kMaxDevices] = {nullptr};

// Device address of g_scratch on `device` (set up once per device, with that
// device current).  Returns GT_OK or GT_ERR_CUDA.
int scratch_address(int device, void **out)
{
    std::lock_guard<std::mutex> lk(g_lock);
    if (!g_addr[device]) {
        int prev = -1;
        if (cudaGetDevice(&prev) != cudaSuccess) return GT_ERR_CUDA;
        if (cudaSetDevice(device) != cudaSuccess) return GT_ERR_CUDA;
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        cudaSetDevice(prev);
        if (e != cudaSuccess || !p) return GT_ERR_CUDA;
        g_addr[device] = p;
    }
    *out = g_addr[device];
    return GT_OK;
}

}  // namespace

extern "C" int avalanche_run_static(gt_ctx *ctx, const gt_run *run, const gt_endpoints *out,
                                    void *stream, gt_stats *stats)
{
    if (!ctx || !run || !out) return GT_ERR_ARG;
    if (run->mode != GT_BATCHED || !run->primaries_on_device) return GT_ERR_ARG;
    if (out->capacity > GT_STATIC_MAX_ELECTRONS || run->n_avalanches > GT_STATIC_MAX_AVALANCHES)
        return GT_ERR_WORKSPACE;
    const int device = gt::context_device(ctx);
    if (device < 0 || device >= kMaxDevices) return GT_ERR_ARG;
    size_t need = 0;
    int rc = gt_workspace_bytes(ctx, run, out->capacity, &need);
    if (rc != GT_OK) return rc;
    if (need > kStaticBytes) return GT_ERR_WORKSPACE;
    void *scratch = nullptr;
    if ((rc = scratch_address(device, &scratch)) != GT_OK) return rc;
    // avalanche_run clears everything that must start at zero (queue flags,
    // header, counters) before its kernels run, so the previous call's
    // contents do not matter.
    return avalanche_run(ctx, run, out, scratch, kStaticBytes, stream, stats);
}
