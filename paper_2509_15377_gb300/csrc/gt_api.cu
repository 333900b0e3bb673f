// gt_api.cu -- host runtime behind the C ABI of gt_avalanche.h: context,
// gas-table and field upload (done once, outside the transport, as in the
// paper's Sec. 3.1 and Fig. 3), work-space layout, the batched and plain
// drivers and error mapping.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "gt_avalanche.h"
#include "gt_kernels.cuh"
#include "gt_launch.h"

using namespace gt;

struct gt_ctx {
    int device = -1;
    int sms = 0;
    size_t smem_optin = 0;
    bool has_gas = false, has_field = false;
    DevGas gas{};
    DevField field{};
    double *d_cum64 = nullptr;
    float *d_cum32 = nullptr;
    double *d_band64 = nullptr;
    float *d_band32 = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    Header *h_hdr = nullptr;  // pinned copy of the work-space header
    unsigned long long *d_obs_counts = nullptr;
    size_t obs_counts_cap = 0;
    double *d_obs_partials = nullptr;
    size_t obs_partials_cap = 0;
    // autotuned batched launch shape per [precision][field kind] (0 = none)
    // autotuned launch shapes per [precision][field kind][majorant]
    // [precision][field kind][majorant][kernel build: basic, general gas,
    // sub-steps/crossings/signals, crossings alone, signals alone]
    int tuned_block[2][5][2][5] = {};
    int tuned_k[2][5][2][5] = {};
    int tuned_m[2][5][2][5] = {};
    // MESH field: element records and search bins (device, owned)
    float *d_tet32 = nullptr;
    double *d_tet64 = nullptr;
    int *d_tet_nb = nullptr;
    int *d_bin_start = nullptr, *d_bin_tets = nullptr;
    // counts gas_table_upload and field_setup calls that replaced device
    // tables: a captured graph holds the tables of its own setup
    unsigned long long setup_gen = 0;
    char last_error[256] = {0};
};

namespace {
// The seed and its Philox round keys: (k0, k1) = (seed_lo, seed_hi) advanced
// by the Weyl constants 0x9E3779B9, 0xBB67AE85 after each of the ten rounds.
static void set_seed(RunParams &p, uint64_t seed)
{
    p.seed = seed;
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        p.rk[2 * r] = k0;
        p.rk[2 * r + 1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// Makes the context's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = false;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

int cuda_fail(gt_ctx *ctx, cudaError_t e, const char *where)
{
    if (ctx)
        snprintf(ctx->last_error, sizeof(ctx->last_error), "%s: %s", where,
                 cudaGetErrorString(e));
    return GT_ERR_CUDA;
}

#define GT_CUDA(ctx, call)                                                                 \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);                         \
    } while (0)

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Work-space layout.  Every region starts on a 256-byte boundary.
struct Layout {
    size_t hdr, ready, bvx, bvy, bvz, belem, created, afield, prim, order, stacks, total;
    size_t stack_entry_bytes;
};

constexpr size_t kStackEntry = 7 * sizeof(double) + 2 * sizeof(uint32_t) + sizeof(uint64_t) +
                               sizeof(int64_t) + sizeof(int32_t);

Layout layout_for(const gt_run *run, int64_t capacity)
{
    Layout L{};
    size_t off = 0;
    L.hdr = off; off = align256(off + sizeof(Header));
    L.ready = off; off = align256(off + sizeof(uint32_t) * (size_t)capacity);
    L.bvx = off; off = align256(off + sizeof(double) * (size_t)capacity);
    L.bvy = off; off = align256(off + sizeof(double) * (size_t)capacity);
    L.bvz = off; off = align256(off + sizeof(double) * (size_t)capacity);
    L.belem = off; off = align256(off + sizeof(int32_t) * (size_t)capacity);
    const size_t na = (size_t)std::max(run->n_avalanches, 1);
    L.created = off; off = align256(off + sizeof(unsigned long long) * na);
    L.afield = off;
    if (!run->primaries_on_device && run->aval_field) off = align256(off + sizeof(double) * na);
    L.prim = off;
    const size_t np = (size_t)std::max<int64_t>(run->n_primaries, 1);
    if (!run->primaries_on_device)
        off = align256(off + np * (8 * sizeof(double) + sizeof(int32_t) + sizeof(uint64_t)) + 8 * 256);
    L.order = off;
    L.stacks = off;
    L.stack_entry_bytes = kStackEntry;
    if (run->mode == GT_PLAIN) {
        off = align256(off + sizeof(long long) * np);
        L.stacks = off;
        off = align256(off + 3 * (kStackEntry * (size_t)capacity + 16 * 256));
    }
    L.total = off;
    return L;
}

// Carve one plain-mode stack (SoA) out of a region.
Stack carve_stack(char *&p, int64_t cap)
{
    Stack s;
    auto take = [&](size_t bytes) {
        char *q = p;
        p += align256(bytes);
        return q;
    };
    s.x = (double *)take(sizeof(double) * cap);
    s.y = (double *)take(sizeof(double) * cap);
    s.z = (double *)take(sizeof(double) * cap);
    s.t = (double *)take(sizeof(double) * cap);
    s.vx = (double *)take(sizeof(double) * cap);
    s.vy = (double *)take(sizeof(double) * cap);
    s.vz = (double *)take(sizeof(double) * cap);
    s.nf = (uint32_t *)take(sizeof(uint32_t) * cap);
    s.nreal = (uint32_t *)take(sizeof(uint32_t) * cap);
    s.uid = (uint64_t *)take(sizeof(uint64_t) * cap);
    s.slot = (int64_t *)take(sizeof(int64_t) * cap);
    s.alive = (int32_t *)take(sizeof(int32_t) * cap);
    return s;
}

int default_block(int precision) { return precision == GT_FP64 ? 256 : 512; }

// Which build of the mixed kernels a run uses (their launch shapes are tuned
// apart): 0 the basic gas, 1 the general gas (anisotropy, attachment, a
// sharing law), 2 sub-steps, crossings or signals (any gas).
int run_variant(const gt_ctx *ctx, const gt_run *r)
{
    const bool signal = r->signal_kind != GT_W_NONE && r->signal_bins > 0;
    // crossings alone and signals alone have builds of their own (mixed)
    if (r->crossing && r->substeps <= 1 && !signal) return 3;
    if (signal && r->substeps <= 1 && !r->crossing) return 4;
    if (r->substeps > 1 || r->crossing || signal) return 2;
    return ctx->gas.any_special ? 1 : 0;
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

}  // namespace

int gt::context_device(const gt_ctx *ctx) { return ctx ? ctx->device : -1; }

extern "C" {

int gt_abi_version(void) { return GT_ABI_VERSION; }

const char *gt_strerror(int code)
{
    switch (code) {
    case GT_OK: return "ok";
    case GT_ERR_ARG: return "invalid argument";
    case GT_ERR_STATE: return "gas table or field not set up";
    case GT_ERR_WORKSPACE: return "work space too small or misaligned";
    case GT_ERR_QUEUE_OVERFLOW: return "endpoint capacity exceeded (result partial)";
    case GT_ERR_TIMEOUT: return "bounded wait or time budget exceeded (result partial)";
    case GT_ERR_CUDA: return "CUDA runtime error";
    case GT_ERR_NO_DEVICE: return "no usable sm_103 CUDA device";
    case GT_ERR_UNSUPPORTED: return "unsupported combination";
    case GT_ERR_HOST_MEMORY: return "host allocation failed";
    default: return "unknown error";
    }
}

const char *gt_last_cuda_error(gt_ctx *ctx) { return ctx ? ctx->last_error : ""; }

int gt_create(gt_ctx **out, int device)
{
    if (!out) return GT_ERR_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n <= 0) {
        cudaGetLastError();
        return GT_ERR_NO_DEVICE;
    }
    if (device < 0 || device >= n) return GT_ERR_NO_DEVICE;
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return GT_ERR_NO_DEVICE;
    if (prop.major * 10 + prop.minor != 103) return GT_ERR_NO_DEVICE;
    gt_ctx *ctx = new (std::nothrow) gt_ctx();
    if (!ctx) return GT_ERR_CUDA;
    ctx->device = device;
    ctx->sms = prop.multiProcessorCount;
    ctx->smem_optin = prop.sharedMemPerBlockOptin;
    DeviceGuard g(device);
    if (!g.ok || configure_fp64(ctx->smem_optin) != cudaSuccess ||
        configure_mixed(ctx->smem_optin) != cudaSuccess ||
        cudaEventCreate(&ctx->ev0) != cudaSuccess || cudaEventCreate(&ctx->ev1) != cudaSuccess ||
        cudaMallocHost((void **)&ctx->h_hdr, sizeof(Header)) != cudaSuccess) {
        gt_destroy(ctx);
        return GT_ERR_CUDA;
    }
    *out = ctx;
    return GT_OK;
}

int gt_abi_sizes(size_t *sizes, int n)
{
    if (!sizes || n < 5) return GT_ERR_ARG;
    sizes[0] = sizeof(gt_gas);
    sizes[1] = sizeof(gt_field);
    sizes[2] = sizeof(gt_run);
    sizes[3] = sizeof(gt_endpoints);
    sizes[4] = sizeof(gt_stats);
    return GT_OK;
}

int gt_destroy(gt_ctx *ctx)
{
    if (!ctx) return GT_OK;
    {
        DeviceGuard g(ctx->device);
        if (ctx->d_cum64) cudaFree(ctx->d_cum64);
        if (ctx->d_cum32) cudaFree(ctx->d_cum32);
        if (ctx->d_band64) cudaFree(ctx->d_band64);
        if (ctx->d_band32) cudaFree(ctx->d_band32);
        if (ctx->d_obs_counts) cudaFree(ctx->d_obs_counts);
        if (ctx->d_obs_partials) cudaFree(ctx->d_obs_partials);
        if (ctx->d_tet32) cudaFree(ctx->d_tet32);
        if (ctx->d_tet64) cudaFree(ctx->d_tet64);
        if (ctx->d_tet_nb) cudaFree(ctx->d_tet_nb);
        if (ctx->d_bin_start) cudaFree(ctx->d_bin_start);
        if (ctx->d_bin_tets) cudaFree(ctx->d_bin_tets);
        if (ctx->ev0) cudaEventDestroy(ctx->ev0);
        if (ctx->ev1) cudaEventDestroy(ctx->ev1);
        if (ctx->h_hdr) cudaFreeHost(ctx->h_hdr);
    }
    delete ctx;
    return GT_OK;
}

static int gas_table_upload_impl(gt_ctx *ctx, const gt_gas *g);
static int field_setup_impl(gt_ctx *ctx, const gt_field *f);
static int avalanche_run_impl(gt_ctx *ctx, const gt_run *r, const gt_endpoints *o, void *ws,
                              size_t ws_bytes, void *stream, gt_stats *stats);

// The entry points that build host-side tables catch a failed host
// allocation: nothing throws across the C ABI.
int gas_table_upload(gt_ctx *ctx, const gt_gas *g)
{
    try {
        return gas_table_upload_impl(ctx, g);
    } catch (const std::bad_alloc &) {
        return GT_ERR_HOST_MEMORY;
    }
}

int field_setup(gt_ctx *ctx, const gt_field *f)
{
    try {
        return field_setup_impl(ctx, f);
    } catch (const std::bad_alloc &) {
        return GT_ERR_HOST_MEMORY;
    }
}

int avalanche_run(gt_ctx *ctx, const gt_run *r, const gt_endpoints *o, void *ws, size_t ws_bytes,
                  void *stream, gt_stats *stats)
{
    try {
        return avalanche_run_impl(ctx, r, o, ws, ws_bytes, stream, stats);
    } catch (const std::bad_alloc &) {
        return GT_ERR_HOST_MEMORY;
    }
}

static int gas_table_upload_impl(gt_ctx *ctx, const gt_gas *g)
{
    if (!ctx || !g) return GT_ERR_ARG;
    const int L = g->n_levels, N = g->n_nodes;
    if (L < 1 || L > GT_MAX_LEVELS || N < 2 || N > (1 << 22) || !finite_pos(g->d_eps) ||
        !g->level_type ||
        !g->threshold || !g->rate || !(g->recoil >= 0.0 && g->recoil < 0.5))
        return GT_ERR_ARG;
    for (int j = 0; j < L; ++j) {
        const int t = g->level_type[j];
        if (t != GT_LEVEL_ELASTIC && t != GT_LEVEL_EXCITATION && t != GT_LEVEL_IONISATION &&
            t != GT_LEVEL_ATTACHMENT)
            return GT_ERR_ARG;
        if (!(g->threshold[j] >= 0.0) || !std::isfinite(g->threshold[j])) return GT_ERR_ARG;
        if (g->xi0 && !(g->xi0[j] > -1.0 && g->xi0[j] < 1.0)) return GT_ERR_ARG;
        if (g->screen && (!(g->screen[j] >= 0.0) || !std::isfinite(g->screen[j])))
            return GT_ERR_ARG;
    }
    if (!(g->split_w >= 0.0) || !std::isfinite(g->split_w)) return GT_ERR_ARG;
    // cumulative rates over levels at every node, FP64, and their maximum
    std::vector<double> cum((size_t)N * L);
    double top = 0.0;
    for (int k = 0; k < N; ++k) {
        double s = 0.0;
        for (int j = 0; j < L; ++j) {
            const double r = g->rate[(size_t)k * L + j];
            if (!(r >= 0.0) || !std::isfinite(r)) return GT_ERR_ARG;
            s += r;
            cum[(size_t)k * L + j] = s;
        }
        top = std::max(top, s);
    }
    const double nu_max = g->nu_max > 0.0 ? g->nu_max : top * (1.0 + 1e-6);
    if (!finite_pos(nu_max) || nu_max < top) return GT_ERR_ARG;
    std::vector<float> cum32(cum.size());
    for (size_t i = 0; i < cum.size(); ++i) cum32[i] = (float)cum[i];

    // Banded majorant: band b spans nodes b*n .. (b+1)*n; its bound is the
    // largest node value of the total rate (linear between nodes), or
    // top * 2^-40 where that is zero, so every window stays finite.  Range
    // maxima over 2^j consecutive bands, j = 0..J, make any band range two
    // lookups.
    if (!(g->band_width >= 0.0) || !std::isfinite(g->band_width)) return GT_ERR_ARG;
    const double bw = g->band_width > 0.0 ? g->band_width : 1.0;
    const int bn = std::max(1, (int)std::floor(bw / g->d_eps + 0.5));
    const int B = std::max(1, (N - 1 + bn - 1) / bn);
    int J = 0;
    while ((2 << J) <= B) ++J;
    std::vector<double> band((size_t)(J + 1) * B);
    for (int b = 0; b < B; ++b) {
        double m = 0.0;
        for (int k = b * bn; k <= (b + 1) * bn && k < N; ++k)
            m = std::max(m, cum[(size_t)k * L + L - 1]);
        band[b] = m > 0.0 ? m : std::ldexp(top, -40);
    }
    for (int j = 1; j <= J; ++j)
        for (int b = 0; b < B; ++b) {
            const int o = b + (1 << (j - 1));
            band[(size_t)j * B + b] = o < B ? std::max(band[(size_t)(j - 1) * B + b],
                                                       band[(size_t)(j - 1) * B + o])
                                            : band[(size_t)(j - 1) * B + b];
        }
    std::vector<float> band32(band.size());
    for (size_t i = 0; i < band.size(); ++i) band32[i] = (float)band[i];

    DeviceGuard dg(ctx->device);
    if (!dg.ok) return GT_ERR_CUDA;
    if (ctx->d_cum64) cudaFree(ctx->d_cum64);
    if (ctx->d_cum32) cudaFree(ctx->d_cum32);
    if (ctx->d_band64) cudaFree(ctx->d_band64);
    if (ctx->d_band32) cudaFree(ctx->d_band32);
    ctx->d_cum64 = nullptr;
    ctx->d_cum32 = nullptr;
    ctx->d_band64 = nullptr;
    ctx->d_band32 = nullptr;
    ctx->has_gas = false;
    GT_CUDA(ctx, cudaMalloc((void **)&ctx->d_cum64, sizeof(double) * cum.size()));
    GT_CUDA(ctx, cudaMalloc((void **)&ctx->d_cum32, sizeof(float) * cum.size()));
    GT_CUDA(ctx, cudaMalloc((void **)&ctx->d_band64, sizeof(double) * band.size()));
    GT_CUDA(ctx, cudaMalloc((void **)&ctx->d_band32, sizeof(float) * band.size()));
    GT_CUDA(ctx, cudaMemcpy(ctx->d_cum64, cum.data(), sizeof(double) * cum.size(),
                            cudaMemcpyHostToDevice));
    GT_CUDA(ctx, cudaMemcpy(ctx->d_cum32, cum32.data(), sizeof(float) * cum.size(),
                            cudaMemcpyHostToDevice));
    GT_CUDA(ctx, cudaMemcpy(ctx->d_band64, band.data(), sizeof(double) * band.size(),
                            cudaMemcpyHostToDevice));
    GT_CUDA(ctx, cudaMemcpy(ctx->d_band32, band32.data(), sizeof(float) * band.size(),
                            cudaMemcpyHostToDevice));
    DevGas &d = ctx->gas;
    d = DevGas{};
    d.n_levels = L;
    d.n_nodes = N;
    d.d_eps = g->d_eps;
    d.inv_d_eps = 1.0 / g->d_eps;
    d.nu_max = nu_max;
    d.inv_nu_max = 1.0 / nu_max;
    d.recoil = g->recoil;
    d.inv_d_eps_f = (float)d.inv_d_eps;
    d.nu_max_f = (float)nu_max;
    d.inv_nu_max_f = (float)d.inv_nu_max;
    d.recoil_f = (float)g->recoil;
    d.last_x_f = (float)(N - 1);
    d.lastk_f = (float)(N - 2);
    d.cum64 = ctx->d_cum64;
    d.cum32 = ctx->d_cum32;
    d.n_bands = B;
    d.band_levels = J + 1;
    // non-decreasing band bounds (a rising total rate): the largest bound
    // over a band range is its top band's, one lookup
    d.bands_monotone = 1;
    for (int b = 1; b < B; ++b)
        if (band[b] < band[b - 1]) d.bands_monotone = 0;
    d.inv_band_width = 1.0 / (bn * g->d_eps);
    d.inv_band_width_f = (float)d.inv_band_width;
    d.last_band_f = (float)(B - 1);
    d.band64 = ctx->d_band64;
    d.band32 = ctx->d_band32;
    d.any_aniso = 0;
    for (int j = 0; j < L; ++j) {
        d.type[j] = g->level_type[j];
        d.thr[j] = g->threshold[j];
        d.xi0[j] = g->xi0 ? g->xi0[j] : 0.0;
        d.screen[j] = g->screen ? g->screen[j] : 0.0;
        if (d.xi0[j] != 0.0 || d.screen[j] > 0.0) d.any_aniso = 1;
    }
    d.split_w = g->split_w;
    d.split_w_f = (float)g->split_w;
    d.level0_elastic = g->level_type[0] == GT_LEVEL_ELASTIC ? 1 : 0;
    d.any_special = d.any_aniso || g->split_w > 0.0;
    for (int j = 0; j < L; ++j)
        if (d.type[j] == GT_LEVEL_ATTACHMENT) d.any_special = 1;
    ctx->has_gas = true;
    ++ctx->setup_gen;
    return GT_OK;
}

int gt_gas_nu_max(gt_ctx *ctx, double *nu_max)
{
    if (!ctx || !nu_max) return GT_ERR_ARG;
    if (!ctx->has_gas) return GT_ERR_STATE;
    *nu_max = ctx->gas.nu_max;
    return GT_OK;
}

// MESH: element records (the layout the device reads, see kMeshRec) and a
// uniform grid of bins over the mesh's box, each listing, in ascending
// order, the elements whose bounding box (padded by a hair) meets it.
// Built on the host once per field, then copied to the device.
static int build_mesh(gt_ctx *ctx, const gt_field *f, DevField &d)
{
    const int64_t nn = f->n_mesh_nodes, nt = f->n_tets;
    if (nn < 4 || nt < 1 || nt > ((int64_t)1 << 26) || nn > ((int64_t)1 << 30) ||
        !f->mesh_nodes || !f->mesh_tets || !f->mesh_values || !(f->wire_r >= 0.0) ||
        !std::isfinite(f->wire_r))
        return GT_ERR_ARG;
    double lo[3], hi[3];
    for (int k = 0; k < 3; ++k) {
        lo[k] = INFINITY;
        hi[k] = -INFINITY;
    }
    double emax = 0.0;
    for (int64_t i = 0; i < nn; ++i) {
        for (int k = 0; k < 3; ++k) {
            const double x = f->mesh_nodes[3 * i + k];
            if (!std::isfinite(x)) return GT_ERR_ARG;
            lo[k] = std::min(lo[k], x);
            hi[k] = std::max(hi[k], x);
        }
        const float *v = f->mesh_values + 4 * i;
        for (int k = 0; k < 4; ++k)
            if (!std::isfinite(v[k])) return GT_ERR_ARG;
        emax = std::max(emax, std::sqrt((double)v[0] * v[0] + (double)v[1] * v[1] +
                                        (double)v[2] * v[2]));
    }
    double ext[3], mean_ext[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < 3; ++k) {
        ext[k] = hi[k] - lo[k];
        if (!(ext[k] > 0.0)) return GT_ERR_ARG;
    }
    std::vector<double> rec(kMeshRec * (size_t)nt, 0.0);
    std::vector<double> box(6 * (size_t)nt);
    for (int64_t t = 0; t < nt; ++t) {
        const int32_t *q = f->mesh_tets + 4 * t;
        const double *v[4];
        const float *val[4];
        for (int i = 0; i < 4; ++i) {
            if (q[i] < 0 || q[i] >= nn) return GT_ERR_ARG;
            v[i] = f->mesh_nodes + 3 * (int64_t)q[i];
            val[i] = f->mesh_values + 4 * (int64_t)q[i];
        }
        double e[3][3], len = 0.0;
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) {
                e[i][k] = v[i + 1][k] - v[0][k];
                len = std::max(len, std::fabs(e[i][k]));
            }
        // rows of the inverse of [e0 e1 e2] (columns): (e1 x e2, e2 x e0, e0 x e1) / det
        double c[3][3];
        for (int i = 0; i < 3; ++i) {
            const double *a = e[(i + 1) % 3], *b = e[(i + 2) % 3];
            c[i][0] = a[1] * b[2] - a[2] * b[1];
            c[i][1] = a[2] * b[0] - a[0] * b[2];
            c[i][2] = a[0] * b[1] - a[1] * b[0];
        }
        const double det = e[0][0] * c[0][0] + e[0][1] * c[0][1] + e[0][2] * c[0][2];
        if (!(std::fabs(det) > 1e-12 * len * len * len)) return GT_ERR_ARG;
        double *r = rec.data() + kMeshRec * t;
        for (int k = 0; k < 3; ++k) r[k] = v[0][k];
        double m[3][3], tx[3];
        for (int k = 0; k < 3; ++k) {  // the element's extent along each axis
            double a = v[0][k], b = v[0][k];
            for (int i = 1; i < 4; ++i) {
                a = std::min(a, v[i][k]);
                b = std::max(b, v[i][k]);
            }
            tx[k] = b - a;
        }
        // FP32 margin: with u = 2^-23, a coordinate l_i = M_i (r - v0) computed
        // from the FP32 position, node and record errs by at most
        // u sum_k |M_ik| (2 |v0_k| + 3 extent_k); l_0 by the sum of those;
        // twice the largest, plus a few roundings of l itself
        const double u = 1.1920928955078125e-7;
        double err0 = 3.0 * u, errmax = 0.0;
        for (int i = 0; i < 3; ++i) {
            double ei = 0.0;
            for (int k = 0; k < 3; ++k) {
                m[i][k] = c[i][k] / det;
                r[4 + 4 * i + k] = m[i][k];
                ei += std::fabs(m[i][k]) * u * (2.0 * std::fabs(v[0][k]) + 3.0 * tx[k]);
            }
            err0 += ei;
            errmax = std::max(errmax, ei);
        }
        r[3] = 2.0 * (std::max(errmax, err0) + 4.0 * u);
        // value at v0 and gradient of each component: sum_i (V_{i+1} - V_0) M_row_i
        for (int comp = 0; comp < 4; ++comp) {
            double g[3] = {0.0, 0.0, 0.0};
            for (int i = 0; i < 3; ++i) {
                const double dv = (double)val[i + 1][comp] - (double)val[0][comp];
                for (int k = 0; k < 3; ++k) g[k] += dv * m[i][k];
            }
            r[16 + comp] = (double)val[0][comp];
            if (comp < 3) {
                for (int k = 0; k < 3; ++k) r[20 + 4 * comp + k] = g[k];
            } else {
                for (int k = 0; k < 3; ++k) r[20 + 4 * k + 3] = g[k];
            }
        }
        for (int k = 0; k < 3; ++k) {
            double a = v[0][k], b = v[0][k];
            for (int i = 1; i < 4; ++i) {
                a = std::min(a, v[i][k]);
                b = std::max(b, v[i][k]);
            }
            box[6 * t + k] = a;
            box[6 * t + 3 + k] = b;
            mean_ext[k] += (b - a) / (double)nt;
        }
    }
    // face neighbours: the faces sorted by their node triple, equal
    // neighbours paired (a face met more than twice is not a mesh)
    std::vector<int> nbr(4 * (size_t)nt, -1);
    {
        struct Face {
            int32_t a, b, c;
            int64_t slot;  // 4 t + the node the face is opposite to
        };
        std::vector<Face> faces(4 * (size_t)nt);
        for (int64_t t = 0; t < nt; ++t)
            for (int i = 0; i < 4; ++i) {
                int32_t n[3], k = 0;
                for (int j = 0; j < 4; ++j)
                    if (j != i) n[k++] = f->mesh_tets[4 * t + j];
                std::sort(n, n + 3);
                faces[4 * t + i] = Face{n[0], n[1], n[2], 4 * t + i};
            }
        std::sort(faces.begin(), faces.end(), [](const Face &x, const Face &y) {
            if (x.a != y.a) return x.a < y.a;
            if (x.b != y.b) return x.b < y.b;
            return x.c < y.c;
        });
        auto same = [](const Face &x, const Face &y) {
            return x.a == y.a && x.b == y.b && x.c == y.c;
        };
        for (size_t i = 0; i < faces.size();) {
            size_t j = i + 1;
            while (j < faces.size() && same(faces[i], faces[j])) ++j;
            if (j - i > 2) return GT_ERR_ARG;
            if (j - i == 2) {
                nbr[faces[i].slot] = (int)(faces[i + 1].slot / 4);
                nbr[faces[i + 1].slot] = (int)(faces[i].slot / 4);
            }
            i = j;
        }
    }
    // bins about half an element's extent per axis, at most 2^24 in all
    int nb[3];
    double total = 1.0;
    for (int k = 0; k < 3; ++k) {
        const double want = mean_ext[k] > 0.0 ? 2.0 * ext[k] / mean_ext[k] : 1.0;
        nb[k] = (int)std::min(std::max(std::ceil(want), 1.0), 1024.0);
        total *= nb[k];
    }
    while (total > (double)(1 << 24)) {
        total = 1.0;
        for (int k = 0; k < 3; ++k) {
            nb[k] = std::max(1, nb[k] / 2);
            total *= nb[k];
        }
    }
    const int64_t ncell = (int64_t)nb[0] * nb[1] * nb[2];
    double h[3], inv[3];
    for (int k = 0; k < 3; ++k) {
        h[k] = ext[k] / nb[k];
        inv[k] = nb[k] / ext[k];
    }
    std::vector<int64_t> count(ncell + 1, 0);
    // an element's box is padded by more than the FP32 rounding of a
    // coordinate, so that an FP32 position falls in a bin that lists it
    double pad[3];
    for (int k = 0; k < 3; ++k)
        pad[k] = std::max(1e-4 * h[k], 4.0 * 1.1920928955078125e-7 *
                                           std::max(std::fabs(lo[k]), std::fabs(hi[k])));
    auto range = [&](int64_t t, int k, int &i0, int &i1) {
        i0 = (int)std::floor((box[6 * t + k] - pad[k] - lo[k]) * inv[k]);
        i1 = (int)std::floor((box[6 * t + 3 + k] + pad[k] - lo[k]) * inv[k]);
        i0 = std::min(std::max(i0, 0), nb[k] - 1);
        i1 = std::min(std::max(i1, 0), nb[k] - 1);
    };
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            for (int64_t c = 0; c < ncell; ++c) count[c + 1] += count[c];
            if (count[ncell] > (int64_t)INT32_MAX) return GT_ERR_ARG;
        }
        std::vector<int64_t> next(pass == 1 ? count.begin() : count.end(), count.end());
        std::vector<int> tets(pass == 1 ? (size_t)count[ncell] : 0);
        for (int64_t t = 0; t < nt; ++t) {
            int a[3], b[3];
            for (int k = 0; k < 3; ++k) range(t, k, a[k], b[k]);
            for (int z = a[2]; z <= b[2]; ++z)
                for (int y = a[1]; y <= b[1]; ++y)
                    for (int x = a[0]; x <= b[0]; ++x) {
                        const int64_t c = ((int64_t)z * nb[1] + y) * nb[0] + x;
                        if (pass == 0)
                            ++count[c + 1];
                        else
                            tets[next[c]++] = (int)t;
                    }
        }
        if (pass == 1) {
            std::vector<int> start(ncell + 1);
            for (int64_t c = 0; c <= ncell; ++c) start[c] = (int)count[c];
            std::vector<float> rec32(rec.size());
            for (size_t i = 0; i < rec.size(); ++i) rec32[i] = (float)rec[i];
            DeviceGuard dg(ctx->device);
            if (!dg.ok) return GT_ERR_CUDA;
            // the new buffers are filled first and replace the context's only
            // then, so that a failure leaves the previous field intact; the
            // holder frees whichever set it ends up with
            struct MeshBuffers {
                float *tet32 = nullptr;
                double *tet64 = nullptr;
                int *nb = nullptr, *start = nullptr, *tets = nullptr;
                ~MeshBuffers()
                {
                    cudaFree(tet32); cudaFree(tet64); cudaFree(nb);
                    cudaFree(start); cudaFree(tets);
                }
            } nbuf;
            GT_CUDA(ctx, cudaMalloc((void **)&nbuf.tet32, sizeof(float) * rec32.size()));
            GT_CUDA(ctx, cudaMalloc((void **)&nbuf.tet64, sizeof(double) * rec.size()));
            GT_CUDA(ctx, cudaMalloc((void **)&nbuf.nb, sizeof(int) * nbr.size()));
            GT_CUDA(ctx, cudaMalloc((void **)&nbuf.start, sizeof(int) * start.size()));
            GT_CUDA(ctx, cudaMalloc((void **)&nbuf.tets,
                                    sizeof(int) * std::max<size_t>(tets.size(), 1)));
            GT_CUDA(ctx, cudaMemcpy(nbuf.tet32, rec32.data(), sizeof(float) * rec32.size(),
                                    cudaMemcpyHostToDevice));
            GT_CUDA(ctx, cudaMemcpy(nbuf.tet64, rec.data(), sizeof(double) * rec.size(),
                                    cudaMemcpyHostToDevice));
            GT_CUDA(ctx, cudaMemcpy(nbuf.nb, nbr.data(), sizeof(int) * nbr.size(),
                                    cudaMemcpyHostToDevice));
            GT_CUDA(ctx, cudaMemcpy(nbuf.start, start.data(), sizeof(int) * start.size(),
                                    cudaMemcpyHostToDevice));
            if (!tets.empty())
                GT_CUDA(ctx, cudaMemcpy(nbuf.tets, tets.data(), sizeof(int) * tets.size(),
                                        cudaMemcpyHostToDevice));
            std::swap(ctx->d_tet32, nbuf.tet32);
            std::swap(ctx->d_tet64, nbuf.tet64);
            std::swap(ctx->d_tet_nb, nbuf.nb);
            std::swap(ctx->d_bin_start, nbuf.start);
            std::swap(ctx->d_bin_tets, nbuf.tets);
        }
    }
    d.tet32 = reinterpret_cast<const float4 *>(ctx->d_tet32);
    d.tet64 = ctx->d_tet64;
    d.tet_nb = reinterpret_cast<const int4 *>(ctx->d_tet_nb);
    d.bin_start = ctx->d_bin_start;
    d.bin_tets = ctx->d_bin_tets;
    for (int k = 0; k < 3; ++k) {
        d.origin[k] = lo[k];
        d.hi[k] = hi[k];
        d.bin_n[k] = nb[k];
        d.bin_lo[k] = lo[k];
        d.bin_inv[k] = inv[k];
        d.bin_lo_f[k] = (float)lo[k];
        d.bin_inv_f[k] = (float)inv[k];
    }
    d.wire_r2 = f->wire_r * f->wire_r;
    if (f->wire_r > 0.0 && f->tube_r > f->wire_r) {
        d.ln_tube = std::log(f->tube_r);
        d.inv_ln_ab = 1.0 / std::log(f->wire_r / f->tube_r);
    }
    d.emax = emax;
    return GT_OK;
}

static int field_setup_impl(gt_ctx *ctx, const gt_field *f)
{
    if (!ctx || !f) return GT_ERR_ARG;
    DevField d{};
    d.kind = f->kind;
    for (int i = 0; i < 3; ++i) {
        if (!std::isfinite(f->b[i])) return GT_ERR_ARG;
        d.w[i] = -kOmega * f->b[i];
    }
    d.has_b = (f->b[0] != 0.0 || f->b[1] != 0.0 || f->b[2] != 0.0) ? 1 : 0;
    d.e0 = f->e0;
    switch (f->kind) {
    case GT_FIELD_UNIFORM:
        if (!std::isfinite(f->e0)) return GT_ERR_ARG;
        break;
    case GT_FIELD_PLATE:
        if (!std::isfinite(f->e0) || !finite_pos(f->gap)) return GT_ERR_ARG;
        d.gap = f->gap;
        d.inv_gap = 1.0 / f->gap;
        break;
    case GT_FIELD_COAX:
        if (!finite_pos(f->wire_r) || !finite_pos(f->tube_r) || f->tube_r <= f->wire_r ||
            !std::isfinite(f->voltage))
            return GT_ERR_ARG;
        d.wire_r2 = f->wire_r * f->wire_r;
        d.tube_r2 = f->tube_r * f->tube_r;
        d.coax_k = f->voltage / std::log(f->tube_r / f->wire_r);
        d.emax = std::fabs(d.coax_k) / f->wire_r;
        d.ln_tube = std::log(f->tube_r);
        d.inv_ln_ab = 1.0 / std::log(f->wire_r / f->tube_r);
        break;
    case GT_FIELD_GRID:
        if (f->nx < 2 || f->ny < 2 || f->nz < 2 || f->nx > (1 << 22) || f->ny > (1 << 22) ||
            f->nz > (1 << 22) || !f->grid ||
            ((uintptr_t)f->grid & 15u) != 0 || !(f->wire_r >= 0.0))
            return GT_ERR_ARG;
        d.nx = f->nx; d.ny = f->ny; d.nz = f->nz;
        for (int i = 0; i < 3; ++i) {
            if (!finite_pos(f->spacing[i]) || !std::isfinite(f->origin[i])) return GT_ERR_ARG;
            d.origin[i] = f->origin[i];
            d.inv_spacing[i] = 1.0 / f->spacing[i];
        }
        d.hi[0] = f->origin[0] + (f->nx - 1) * f->spacing[0];
        d.hi[1] = f->origin[1] + (f->ny - 1) * f->spacing[1];
        d.hi[2] = f->origin[2] + (f->nz - 1) * f->spacing[2];
        d.wire_r2 = f->wire_r * f->wire_r;
        d.grid = reinterpret_cast<const float4 *>(f->grid);
        if (f->wire_r > 0.0 && f->tube_r > f->wire_r) {
            d.ln_tube = std::log(f->tube_r);
            d.inv_ln_ab = 1.0 / std::log(f->wire_r / f->tube_r);
        }
        {
            DeviceGuard dg(ctx->device);
            if (!dg.ok) return GT_ERR_CUDA;
            GT_CUDA(ctx, grid_emax(d.grid, (long long)f->nx * f->ny * f->nz, ctx->sms, &d.emax));
        }
        break;
    case GT_FIELD_MESH: {
        const int rc = build_mesh(ctx, f, d);
        if (rc != GT_OK) return rc;
        break;
    }
    default:
        return GT_ERR_ARG;
    }
    // FP32 copies used by the mixed-precision step
    d.e0_f = (float)d.e0;
    d.coax_k_f = (float)d.coax_k;
    for (int i = 0; i < 3; ++i) {
        d.w_f[i] = (float)d.w[i];
        d.origin_f[i] = (float)d.origin[i];
        d.inv_spacing_f[i] = (float)d.inv_spacing[i];
        const double m = 1e-5 * (d.hi[i] - d.origin[i]);
        d.box_lo_f[i] = (float)(d.origin[i] + m);
        d.box_hi_f[i] = (float)(d.hi[i] - m);
    }
    d.cell_hi_f[0] = (float)(d.nx - 2); d.cell_hi_f[1] = (float)(d.ny - 2);
    d.cell_hi_f[2] = (float)(d.nz - 2);
    d.node_hi_f[0] = (float)(d.nx - 1); d.node_hi_f[1] = (float)(d.ny - 1);
    d.node_hi_f[2] = (float)(d.nz - 1);
    d.wire_r2_hi_f = (float)(d.wire_r2 * 1.00001);
    d.tube_r2_lo_f = (float)(d.tube_r2 * 0.99999);
    ctx->field = d;
    ctx->has_field = true;
    ++ctx->setup_gen;
    if (d.kind != GT_FIELD_MESH && ctx->d_tet32) {  // a previous mesh is no longer used
        DeviceGuard dg(ctx->device);
        cudaFree(ctx->d_tet32); cudaFree(ctx->d_tet64); cudaFree(ctx->d_tet_nb);
        cudaFree(ctx->d_bin_start); cudaFree(ctx->d_bin_tets);
        ctx->d_tet32 = nullptr; ctx->d_tet64 = nullptr; ctx->d_tet_nb = nullptr;
        ctx->d_bin_start = nullptr; ctx->d_bin_tets = nullptr;
    }
    return GT_OK;
}

int gt_workspace_bytes(gt_ctx *ctx, const gt_run *run, int64_t capacity, size_t *bytes)
{
    if (!ctx || !run || !bytes || capacity < 0 || run->n_avalanches < 0 || run->n_primaries < 0)
        return GT_ERR_ARG;
    *bytes = layout_for(run, capacity).total;
    return GT_OK;
}

// ------------------------------------------------------------------ run
static int validate_run(gt_ctx *ctx, const gt_run *r, const gt_endpoints *o, void *ws,
                        size_t ws_bytes)
{
    if (!r || !o) return GT_ERR_ARG;
    if (!ctx->has_gas || !ctx->has_field) return GT_ERR_STATE;
    if (r->n_primaries < 0 || r->n_avalanches < 0) return GT_ERR_ARG;
    if (r->n_primaries > 0 && r->n_avalanches < 1) return GT_ERR_ARG;
    if (r->aval_base < 0 || (int64_t)r->aval_base + r->n_avalanches > INT32_MAX) return GT_ERR_ARG;
    if (r->precision != GT_FP64 && r->precision != GT_MIXED) return GT_ERR_ARG;
    if (r->mode != GT_BATCHED && r->mode != GT_PLAIN) return GT_ERR_ARG;
    if (!std::isfinite(r->t_max)) return GT_ERR_ARG;
    if (r->block < 0 || r->refill_period < 0 || r->grid < 0 || r->flights_per_phase < 0)
        return GT_ERR_ARG;
    if ((r->majorant != GT_MAJORANT_GLOBAL && r->majorant != GT_MAJORANT_BANDED) ||
        !(r->majorant_window >= 0.0) || !std::isfinite(r->majorant_window) ||
        r->substeps < 0 || r->substeps > 4096 || (r->crossing != 0 && r->crossing != 1))
        return GT_ERR_ARG;
    if (r->signal_kind < GT_W_NONE || r->signal_kind > GT_W_MAP) return GT_ERR_ARG;
    if (r->signal_kind != GT_W_NONE) {
        const int k = ctx->field.kind;
        if (r->signal_bins < 0 || !(r->signal_dt > 0.0) || !std::isfinite(r->signal_dt) ||
            !std::isfinite(r->signal_t0) ||
            (r->signal_kind == GT_W_PLATE && k != GT_FIELD_PLATE) ||
            (r->signal_kind == GT_W_COAX && k != GT_FIELD_COAX && k != GT_FIELD_GRID &&
             k != GT_FIELD_MESH) ||
            (r->signal_kind == GT_W_MAP && k != GT_FIELD_GRID && k != GT_FIELD_MESH))
            return GT_ERR_ARG;
        if (r->signal_bins > 0 && r->n_avalanches > 0 && !o->signal) return GT_ERR_ARG;
        if (r->signal_kind == GT_W_COAX && ctx->field.inv_ln_ab == 0.0) return GT_ERR_ARG;
    }
    if (r->block && (r->block % 32 != 0 ||
                     r->block > (r->precision == GT_FP64 ? max_block_fp64() : max_block_mixed())))
        return GT_ERR_ARG;
    if (r->spin_limit_ms < 0 || r->time_limit_ms < 0) return GT_ERR_ARG;
    // an electron in the unbounded uniform field must stop somehow
    if (ctx->field.kind == GT_FIELD_UNIFORM && !(r->t_max > 0.0) && r->coll_limit == 0)
        return GT_ERR_ARG;
    const int64_t need = r->n_primaries + ((r->debug_flags & GT_DEBUG_UNFILLED_SLOT) ? 1 : 0);
    if (o->capacity < need || o->capacity < 0) return GT_ERR_ARG;
    if (o->capacity > 0 && (!o->x0 || !o->y0 || !o->z0 || !o->t0 || !o->e0 || !o->x1 || !o->y1 ||
                            !o->z1 || !o->t1 || !o->e1 || !o->status || !o->aval || !o->uid ||
                            !o->n_flight))
        return GT_ERR_ARG;
    if (r->n_avalanches > 0 && (!o->electrons || !o->tallies)) return GT_ERR_ARG;
    if (r->n_primaries > 0 && (!r->x || !r->y || !r->z || !r->t || !r->e || !r->dx || !r->dy ||
                               !r->dz || !r->aval || !r->uid))
        return GT_ERR_ARG;
    if (!ws || ((uintptr_t)ws & 255u) != 0) return GT_ERR_WORKSPACE;
    if (ws_bytes < layout_for(r, o->capacity).total) return GT_ERR_WORKSPACE;
    if (!r->primaries_on_device) {
        for (int64_t i = 0; i < r->n_primaries; ++i) {
            if (r->aval[i] < 0 || r->aval[i] >= r->n_avalanches) return GT_ERR_ARG;
            if (!(r->e[i] >= 0.0) || !std::isfinite(r->e[i])) return GT_ERR_ARG;
        }
    }
    return GT_OK;
}

static int finish_status(const Header &h)
{
    if (h.error & ERR_BADARG) return GT_ERR_ARG;
    if (h.error & ERR_TIMEOUT) return GT_ERR_TIMEOUT;
    if (h.error & ERR_OVERFLOW) return GT_ERR_QUEUE_OVERFLOW;
    return GT_OK;
}

// A run's parameters and launch shape, decided on the host.
struct RunPlan {
    RunParams p{};
    SeedArgs sa{};
    int block = 0, grid = 0;
    size_t smem = 0;
    bool fp64 = false, smem_table = false;
};

// Fills the plan of a validated run.  Host primaries are staged into the
// work space with copies on stream s (the only device work here).
static int plan_run(gt_ctx *ctx, const gt_run *r, const gt_endpoints *o, void *ws,
                    cudaStream_t s, RunPlan &pl)
{
    const Layout Ly = layout_for(r, o->capacity);
    char *base = static_cast<char *>(ws);
    const int64_t np = r->n_primaries;
    const int na = r->n_avalanches;
    const int L = ctx->gas.n_levels;
    RunParams &p = pl.p;
    SeedArgs &sa = pl.sa;
    p.gas = ctx->gas;
    p.field = ctx->field;
    p.x0 = o->x0; p.y0 = o->y0; p.z0 = o->z0; p.t0 = o->t0; p.e0 = o->e0;
    p.x1 = o->x1; p.y1 = o->y1; p.z1 = o->z1; p.t1 = o->t1; p.e1 = o->e1;
    p.status = o->status; p.aval = o->aval; p.uid = o->uid; p.nflight = o->n_flight;
    p.tallies = o->tallies; p.electrons = o->electrons;
    p.capacity = o->capacity;
    p.hdr = reinterpret_cast<Header *>(base + Ly.hdr);
    p.ready = reinterpret_cast<unsigned int *>(base + Ly.ready);
    p.bvx = reinterpret_cast<double *>(base + Ly.bvx);
    p.bvy = reinterpret_cast<double *>(base + Ly.bvy);
    p.bvz = reinterpret_cast<double *>(base + Ly.bvz);
    p.belem = reinterpret_cast<int32_t *>(base + Ly.belem);
    p.created = reinterpret_cast<unsigned long long *>(base + Ly.created);
    set_seed(p, r->seed);
    p.t_max = r->t_max > 0.0 ? r->t_max : 0.0;
    p.coll_limit = r->coll_limit;
    const int prec_i = r->precision == GT_FP64 ? 0 : 1;
    const int maj_i = r->majorant == GT_MAJORANT_BANDED ? 1 : 0;
    const int var_i = run_variant(ctx, r);
    const int tuned_k = ctx->tuned_k[prec_i][ctx->field.kind][maj_i][var_i];
    const int tuned_m = ctx->tuned_m[prec_i][ctx->field.kind][maj_i][var_i];
    p.refill_period = r->refill_period > 0 ? r->refill_period
                                           : (tuned_k > 0 ? tuned_k : (prec_i ? 16 : 32));
    // most banded flights end in a real collision, so a round flies once;
    // with one global nu_max most are null and a round flies several times
    p.flights_per_phase = r->flights_per_phase > 0 ? r->flights_per_phase
                                                   : (tuned_m > 0 ? tuned_m : (maj_i ? 1 : 6));
    p.majorant = r->majorant;
    p.window = r->majorant_window > 0.0 ? r->majorant_window : 2.0;
    p.window_f = (float)p.window;
    p.substeps = r->substeps > 1 ? r->substeps : 1;
    p.crossing = r->crossing;
    // a field re-evaluated along the flight: bound its reach by the largest
    // field of the volume (uniform and plate fields do not change)
    p.field_emax = p.substeps > 1 ? ctx->field.emax : 0.0;
    p.field_emax_f = (float)(p.field_emax * (1.0 + 1e-6));
    p.signal_kind = r->signal_bins > 0 ? r->signal_kind : GT_W_NONE;
    p.signal_bins = p.signal_kind != GT_W_NONE ? r->signal_bins : 0;
    p.signal_t0 = r->signal_t0;
    p.signal_dt = r->signal_dt;
    p.signal_inv_dt = p.signal_bins ? 1.0 / r->signal_dt : 0.0;
    p.signal = p.signal_bins ? o->signal : nullptr;
    p.size_limit = r->size_limit;
    p.spin_limit_ns = (long long)((r->spin_limit_ms > 0 ? r->spin_limit_ms : 60000.0) * 1e6);
    p.time_limit_ns = (long long)((r->time_limit_ms > 0 ? r->time_limit_ms : 600000.0) * 1e6);
    p.n_avalanches = na;
    p.aval_base = r->aval_base;

    // primaries: stage host arrays in the work space (inside the run)
    sa.n = np;
    sa.unfilled_slot = (r->debug_flags & GT_DEBUG_UNFILLED_SLOT) ? 1 : 0;
    p.aval_field = r->aval_field;
    if (!r->primaries_on_device) {
        char *q = base + Ly.prim;
        auto stage = [&](const void *src, size_t bytes) -> void * {
            void *dst = q;
            q += align256(bytes);
            if (bytes && cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
                return nullptr;
            return dst;
        };
        const size_t db = sizeof(double) * (size_t)np;
        void *ptrs[10] = {stage(r->x, db), stage(r->y, db), stage(r->z, db), stage(r->t, db),
                          stage(r->e, db), stage(r->dx, db), stage(r->dy, db), stage(r->dz, db),
                          stage(r->aval, sizeof(int32_t) * (size_t)np),
                          stage(r->uid, sizeof(uint64_t) * (size_t)np)};
        for (void *v : ptrs)
            if (!v) return cuda_fail(ctx, cudaGetLastError(), "primaries upload");
        sa.x = (const double *)ptrs[0]; sa.y = (const double *)ptrs[1];
        sa.z = (const double *)ptrs[2]; sa.t = (const double *)ptrs[3];
        sa.e = (const double *)ptrs[4]; sa.dx = (const double *)ptrs[5];
        sa.dy = (const double *)ptrs[6]; sa.dz = (const double *)ptrs[7];
        sa.aval = (const int32_t *)ptrs[8]; sa.uid = (const uint64_t *)ptrs[9];
        if (r->aval_field) {
            void *af = base + Ly.afield;
            GT_CUDA(ctx, cudaMemcpyAsync(af, r->aval_field, sizeof(double) * (size_t)na,
                                         cudaMemcpyHostToDevice, s));
            p.aval_field = (const double *)af;
        }
    } else {
        sa.x = r->x; sa.y = r->y; sa.z = r->z; sa.t = r->t; sa.e = r->e;
        sa.dx = r->dx; sa.dy = r->dy; sa.dz = r->dz; sa.aval = r->aval; sa.uid = r->uid;
    }

    // outputs and queue flags start from zero
    if (o->capacity > 0)
        GT_CUDA(ctx, cudaMemsetAsync(p.ready, 0, sizeof(uint32_t) * (size_t)o->capacity, s));
    if (na > 0) {
        GT_CUDA(ctx, cudaMemsetAsync(o->tallies, 0, sizeof(uint64_t) * (size_t)na * (L + 1), s));
        if (p.signal_bins)
            GT_CUDA(ctx, cudaMemsetAsync(o->signal, 0,
                                         sizeof(double) * (size_t)na * (size_t)p.signal_bins, s));
        GT_CUDA(ctx, cudaMemsetAsync(o->electrons, 0, sizeof(uint64_t) * (size_t)na, s));
        if (r->size_limit)
            GT_CUDA(ctx, cudaMemsetAsync(p.created, 0, sizeof(unsigned long long) * (size_t)na, s));
    }
    const bool fp64 = r->precision == GT_FP64;
    const int tuned_b = ctx->tuned_block[prec_i][ctx->field.kind][maj_i][var_i];
    const int block = r->block ? r->block
                               : (r->mode == GT_BATCHED && tuned_b > 0 ? tuned_b
                                                                       : default_block(r->precision));
    const int band_entries = ctx->gas.n_bands * ctx->gas.band_levels;
    const size_t smem_tab = shared_bytes(L, ctx->gas.n_nodes, block, true, band_entries);
    const size_t smem_cap = ctx->smem_optin - kStaticSmemReserve;
    const bool smem_table = !fp64 && smem_tab <= smem_cap;
    const size_t smem = shared_bytes(L, ctx->gas.n_nodes, block, smem_table, band_entries);
    if (smem > smem_cap) return GT_ERR_UNSUPPORTED;
    pl.block = block;
    pl.smem = smem;
    pl.fp64 = fp64;
    pl.smem_table = smem_table;
    if (r->mode == GT_BATCHED) {
        const int occ = fp64 ? occupancy_batched_fp64(ctx->field.kind, block, smem)
                             : occupancy_batched_mixed(ctx->field.kind, smem_table, block, smem);
        if (occ < 1) return GT_ERR_UNSUPPORTED;
        pl.grid = r->grid ? r->grid : ctx->sms * occ;
    }
    return GT_OK;
}

// Outputs, queue flags and the run header start from zero; then the
// primaries are seeded.
static int enqueue_start(gt_ctx *ctx, const RunPlan &pl, const gt_endpoints *o, int na,
                         cudaStream_t s)
{
    const RunParams &p = pl.p;
    const int L = ctx->gas.n_levels;
    GT_CUDA(ctx, cudaMemsetAsync(p.hdr, 0, sizeof(Header), s));
    if (o->capacity > 0)
        GT_CUDA(ctx, cudaMemsetAsync(p.ready, 0, sizeof(uint32_t) * (size_t)o->capacity, s));
    if (na > 0) {
        GT_CUDA(ctx, cudaMemsetAsync(o->tallies, 0, sizeof(uint64_t) * (size_t)na * (L + 1), s));
        if (p.signal_bins)
            GT_CUDA(ctx, cudaMemsetAsync(o->signal, 0,
                                         sizeof(double) * (size_t)na * (size_t)p.signal_bins, s));
        GT_CUDA(ctx, cudaMemsetAsync(o->electrons, 0, sizeof(uint64_t) * (size_t)na, s));
        if (p.size_limit)
            GT_CUDA(ctx, cudaMemsetAsync(p.created, 0, sizeof(unsigned long long) * (size_t)na, s));
    }
    GT_CUDA(ctx, launch_seed(p, pl.sa, s));
    return GT_OK;
}

// The rest of a batched run: the persistent transport between ev0 and ev1,
// the per-avalanche electron counts and the header copied to h_hdr.  No
// host synchronisation: the sequence can be captured in a CUDA graph (with
// `capture`, the events become event-record nodes of the graph).
static int enqueue_batched(gt_ctx *ctx, const RunPlan &pl, cudaStream_t s, cudaEvent_t ev0,
                           cudaEvent_t ev1, Header *h_hdr, bool capture = false)
{
    const RunParams &p = pl.p;
    const unsigned evf = capture ? cudaEventRecordExternal : cudaEventRecordDefault;
    GT_CUDA(ctx, cudaEventRecordWithFlags(ev0, s, evf));
    GT_CUDA(ctx, pl.fp64 ? launch_batched_fp64(p, pl.grid, pl.block, pl.smem, s)
                         : launch_batched_mixed(p, pl.smem_table, pl.grid, pl.block, pl.smem, s));
    GT_CUDA(ctx, cudaEventRecordWithFlags(ev1, s, evf));
    GT_CUDA(ctx, launch_count_electrons(p, ctx->sms, s));
    GT_CUDA(ctx, cudaMemcpyAsync(h_hdr, p.hdr, sizeof(Header), cudaMemcpyDeviceToHost, s));
    return GT_OK;
}

static void fill_stats(const Header &h, const RunPlan &pl, int64_t capacity, double transport_ms,
                       int launches, int iterations, int grid, int rc, gt_stats *stats)
{
    if (!stats) return;
    stats->n_endpoints = (int64_t)std::min<unsigned long long>(h.tail, (unsigned long long)capacity);
    stats->n_dropped = (int64_t)h.dropped;
    stats->real_collisions = h.real;
    stats->null_collisions = h.nul;
    stats->flights = h.flights;
    stats->transport_ms = transport_ms;
    stats->launches = launches;
    stats->iterations = iterations;
    stats->status = rc;
    stats->block = pl.block;
    stats->refill_period = pl.p.refill_period;
    stats->grid = grid;
    stats->flights_per_phase = pl.p.flights_per_phase;
}

static int avalanche_run_impl(gt_ctx *ctx, const gt_run *r, const gt_endpoints *o, void *ws,
                              size_t ws_bytes, void *stream, gt_stats *stats)
{
    if (!ctx) return GT_ERR_ARG;
    int rc = validate_run(ctx, r, o, ws, ws_bytes);
    if (rc != GT_OK) return rc;
    DeviceGuard dg(ctx->device);
    if (!dg.ok) return GT_ERR_CUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    RunPlan pl;
    if ((rc = plan_run(ctx, r, o, ws, s, pl)) != GT_OK) return rc;
    const RunParams &p = pl.p;
    const Layout Ly = layout_for(r, o->capacity);
    char *base = static_cast<char *>(ws);
    const int64_t np = r->n_primaries;
    const int na = r->n_avalanches;
    const int L = ctx->gas.n_levels;
    const bool fp64 = pl.fp64;
    const bool smem_table = pl.smem_table;
    const int block = pl.block;
    const int band_entries = ctx->gas.n_bands * ctx->gas.band_levels;
    if ((rc = enqueue_start(ctx, pl, o, na, s)) != GT_OK) return rc;
    int launches = 1;
    int iterations = 0, grid = 0;
    unsigned host_err = 0;  // aborts decided on the host (plain mode)
    double transport_ms = 0.0;

    if (r->mode == GT_BATCHED) {
        grid = pl.grid;
        if ((rc = enqueue_batched(ctx, pl, s, ctx->ev0, ctx->ev1, ctx->h_hdr)) != GT_OK) return rc;
        launches += 2;
        iterations = 1;
        GT_CUDA(ctx, cudaStreamSynchronize(s));
    } else {
        // one avalanche at a time: seed, then generations until none is active
        std::vector<int32_t> av((size_t)np);
        if (np > 0) {
            if (r->primaries_on_device) {
                GT_CUDA(ctx, cudaMemcpyAsync(av.data(), r->aval, sizeof(int32_t) * (size_t)np,
                                             cudaMemcpyDeviceToHost, s));
                GT_CUDA(ctx, cudaStreamSynchronize(s));
            } else {
                std::memcpy(av.data(), r->aval, sizeof(int32_t) * (size_t)np);
            }
        }
        std::vector<long long> first((size_t)na + 1, 0), order((size_t)np);
        for (int64_t i = 0; i < np; ++i)
            if (av[i] >= 0 && av[i] < na) first[av[i] + 1]++;
        for (int a = 0; a < na; ++a) first[a + 1] += first[a];
        {
            std::vector<long long> fill(first.begin(), first.end() - 1);
            for (int64_t i = 0; i < np; ++i)
                if (av[i] >= 0 && av[i] < na) order[fill[av[i]]++] = i;
        }
        long long *d_order = reinterpret_cast<long long *>(base + Ly.order);
        if (np > 0)
            GT_CUDA(ctx, cudaMemcpyAsync(d_order, order.data(), sizeof(long long) * (size_t)np,
                                         cudaMemcpyHostToDevice, s));
        char *sp = base + Ly.stacks;
        Stack st[3] = {carve_stack(sp, o->capacity), carve_stack(sp, o->capacity),
                       carve_stack(sp, o->capacity)};
        const auto t_host0 = std::chrono::steady_clock::now();
        GT_CUDA(ctx, cudaEventRecord(ctx->ev0, s));
        // invalid device-side primaries are caught before any transport
        GT_CUDA(ctx, cudaMemcpyAsync(ctx->h_hdr, p.hdr, sizeof(Header), cudaMemcpyDeviceToHost, s));
        GT_CUDA(ctx, cudaStreamSynchronize(s));
        bool stop = (ctx->h_hdr->error & ERR_BADARG) != 0;
        for (int a = 0; a < na && !stop; ++a) {
            const long long cnt = first[a + 1] - first[a];
            if (cnt == 0) continue;
            GT_CUDA(ctx, cudaMemsetAsync(&p.hdr->n_new[0], 0, 4 * sizeof(unsigned long long), s));
            GT_CUDA(ctx, launch_plain_init(p, st[0], d_order, first[a], cnt, s));
            ++launches;
            int cur = 0, parity = 0;
            long long n_active = cnt;
            while (n_active > 0) {
                PlainArgs pa;
                pa.cur = st[cur];
                pa.fresh = st[2];
                pa.next = st[1 - cur];
                pa.n_active = n_active;
                pa.parity = parity;
                pa.aval = a;
                GT_CUDA(ctx, fp64 ? launch_plain_fp64(p, pa, std::min(block, 128),
                                                      shared_bytes(L, ctx->gas.n_nodes, std::min(block, 128), false, band_entries), s)
                                  : launch_plain_mixed(p, pa, smem_table, std::min(block, 128),
                                                       shared_bytes(L, ctx->gas.n_nodes, std::min(block, 128), smem_table, band_entries), s));
                GT_CUDA(ctx, launch_plain_compact(p, pa, s));
                launches += 2;
                GT_CUDA(ctx, cudaMemcpyAsync(ctx->h_hdr, p.hdr, sizeof(Header),
                                             cudaMemcpyDeviceToHost, s));
                GT_CUDA(ctx, cudaStreamSynchronize(s));
                ++iterations;
                n_active = (long long)ctx->h_hdr->n_next[parity];
                cur = 1 - cur;
                parity ^= 1;
                const double host_ms = std::chrono::duration<double, std::milli>(
                                           std::chrono::steady_clock::now() - t_host0).count();
                if ((ctx->h_hdr->error & (ERR_TIMEOUT | ERR_BADARG)) ||
                    host_ms > (double)p.time_limit_ns * 1e-6) {
                    if (!(ctx->h_hdr->error & ERR_BADARG)) ctx->h_hdr->error |= ERR_TIMEOUT;
                    stop = true;
                    break;
                }
            }
        }
        GT_CUDA(ctx, cudaEventRecord(ctx->ev1, s));
        grid = 0;
        if (stop) host_err = ctx->h_hdr->error & (ERR_TIMEOUT | ERR_BADARG);
    }

    if (r->mode != GT_BATCHED) {
        GT_CUDA(ctx, launch_count_electrons(p, ctx->sms, s));
        ++launches;
        GT_CUDA(ctx, cudaMemcpyAsync(ctx->h_hdr, p.hdr, sizeof(Header), cudaMemcpyDeviceToHost, s));
        GT_CUDA(ctx, cudaStreamSynchronize(s));
    }
    float ms = 0.f;
    GT_CUDA(ctx, cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
    transport_ms = ms;
    Header &h = *ctx->h_hdr;
    h.error |= host_err;
    rc = finish_status(h);
    fill_stats(h, pl, o->capacity, transport_ms, launches, iterations, grid, rc, stats);
    return rc;
}


// ---------------------------------------------------------------- graphs
struct gt_graph {
    gt_ctx *ctx = nullptr;
    RunPlan pl;
    gt_endpoints o{};
    int na = 0;
    cudaStream_t cap = nullptr;    // capture only: nothing runs on it
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr;  // transport start/end, run end
    Header *h_hdr = nullptr;       // pinned, written by the graph's last copy
    uint64_t seed = 0;
    unsigned long long setup_gen = 0;  // the context's setup the graph was recorded with
    bool launched = false;
};

namespace {

void graph_free(gt_graph *g)
{
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->ev0) cudaEventDestroy(g->ev0);
    if (g->ev1) cudaEventDestroy(g->ev1);
    if (g->ev2) cudaEventDestroy(g->ev2);
    if (g->h_hdr) cudaFreeHost(g->h_hdr);
    if (g->cap) cudaStreamDestroy(g->cap);
    delete g;
}

// Records the run's device work into a new graph.
int graph_capture(gt_graph *g, cudaGraph_t *graph)
{
    gt_ctx *ctx = g->ctx;
    GT_CUDA(ctx, cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_start(ctx, g->pl, &g->o, g->na, g->cap);
    if (rc == GT_OK) rc = enqueue_batched(ctx, g->pl, g->cap, g->ev0, g->ev1, g->h_hdr, true);
    if (rc == GT_OK && cudaEventRecordWithFlags(g->ev2, g->cap, cudaEventRecordExternal) !=
                           cudaSuccess)
        rc = cuda_fail(ctx, cudaGetLastError(), "cudaEventRecordWithFlags");
    cudaGraph_t out = nullptr;
    const cudaError_t e = cudaStreamEndCapture(g->cap, &out);
    if (rc != GT_OK) {
        if (out) cudaGraphDestroy(out);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
    *graph = out;
    return GT_OK;
}

}  // namespace

int gt_graph_create(gt_ctx *ctx, const gt_run *run, const gt_endpoints *out, void *ws,
                    size_t ws_bytes, gt_graph **graph)
{
    if (!ctx || !graph) return GT_ERR_ARG;
    *graph = nullptr;
    int rc = validate_run(ctx, run, out, ws, ws_bytes);
    if (rc != GT_OK) return rc;
    if (run->mode != GT_BATCHED || !run->primaries_on_device) return GT_ERR_UNSUPPORTED;
    DeviceGuard dg(ctx->device);
    if (!dg.ok) return GT_ERR_CUDA;
    gt_graph *g = new (std::nothrow) gt_graph();
    if (!g) return GT_ERR_CUDA;
    g->ctx = ctx;
    g->o = *out;
    g->na = run->n_avalanches;
    g->seed = run->seed;
    g->setup_gen = ctx->setup_gen;
    cudaGraph_t gr = nullptr;
    if (cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&g->ev0) != cudaSuccess || cudaEventCreate(&g->ev1) != cudaSuccess ||
        cudaEventCreate(&g->ev2) != cudaSuccess ||
        cudaMallocHost((void **)&g->h_hdr, sizeof(Header)) != cudaSuccess) {
        rc = cuda_fail(ctx, cudaGetLastError(), "gt_graph_create");
    } else {
        rc = plan_run(ctx, run, out, ws, g->cap, g->pl);
    }
    if (rc == GT_OK) rc = graph_capture(g, &gr);
    if (rc == GT_OK) {
        const cudaError_t e = cudaGraphInstantiate(&g->exec, gr, 0);
        if (e != cudaSuccess) rc = cuda_fail(ctx, e, "cudaGraphInstantiate");
    }
    if (gr) cudaGraphDestroy(gr);
    if (rc != GT_OK) {
        graph_free(g);
        return rc;
    }
    *graph = g;
    return GT_OK;
}

int gt_graph_launch(gt_graph *g, uint64_t seed, void *stream)
{
    if (!g) return GT_ERR_ARG;
    gt_ctx *ctx = g->ctx;
    // the gas table or field was set again since the graph was recorded:
    // its kernels would read the replaced (freed) tables
    if (g->setup_gen != ctx->setup_gen) return GT_ERR_STATE;
    DeviceGuard dg(ctx->device);
    if (!dg.ok) return GT_ERR_CUDA;
    if (seed != g->seed) {
        // a new seed: record the run again and update the instantiated graph
        set_seed(g->pl.p, seed);
        cudaGraph_t gr = nullptr;
        int rc = graph_capture(g, &gr);
        if (rc != GT_OK) return rc;
        cudaGraphExecUpdateResultInfo info;
        if (cudaGraphExecUpdate(g->exec, gr, &info) != cudaSuccess) {
            cudaGetLastError();
            cudaGraphExecDestroy(g->exec);
            g->exec = nullptr;
            const cudaError_t e = cudaGraphInstantiate(&g->exec, gr, 0);
            if (e != cudaSuccess) {
                cudaGraphDestroy(gr);
                return cuda_fail(ctx, e, "cudaGraphInstantiate");
            }
        }
        cudaGraphDestroy(gr);
        g->seed = seed;
    }
    GT_CUDA(ctx, cudaGraphLaunch(g->exec, reinterpret_cast<cudaStream_t>(stream)));
    g->launched = true;
    return GT_OK;
}

int gt_graph_stats(gt_graph *g, gt_stats *stats)
{
    if (!g || !stats) return GT_ERR_ARG;
    if (!g->launched) return GT_ERR_STATE;
    gt_ctx *ctx = g->ctx;
    DeviceGuard dg(ctx->device);
    if (!dg.ok) return GT_ERR_CUDA;
    GT_CUDA(ctx, cudaEventSynchronize(g->ev2));
    float ms = 0.f;
    GT_CUDA(ctx, cudaEventElapsedTime(&ms, g->ev0, g->ev1));
    const Header &h = *g->h_hdr;
    const int rc = finish_status(h);
    fill_stats(h, g->pl, g->o.capacity, ms, 3, 1, g->pl.grid, rc, stats);
    return rc;
}

int gt_graph_destroy(gt_graph *g)
{
    if (!g) return GT_OK;
    DeviceGuard dg(g->ctx->device);
    graph_free(g);
    return GT_OK;
}

int gt_autotune(gt_ctx *ctx, const gt_run *run, const gt_endpoints *out, void *ws,
                size_t ws_bytes, void *stream, gt_tune_point *points, int32_t max_points,
                int32_t *n_points, gt_tune_point *best)
{
    if (!ctx || !run || !best) return GT_ERR_ARG;
    gt_run r = *run;
    r.mode = GT_BATCHED;
    const bool fp64 = r.precision == GT_FP64;
    // candidate values per dimension: threads per CTA, refill period,
    // flights per phase (mixed only); a dimension the caller set is fixed
    static const int blocks_mixed[] = {512, 768, 896, 1024};
    static const int blocks_fp64[] = {128, 256, 512};
    static const int ks_mixed[] = {4, 8, 16, 32};
    static const int ks_fp64[] = {8, 16, 32, 64};
    static const int ms_mixed[] = {1, 2, 4, 6};
    static const int ms_fp64[] = {1};
    std::vector<int> cand[3];
    if (run->block > 0) cand[0] = {run->block};
    else if (fp64) cand[0].assign(blocks_fp64, blocks_fp64 + 3);
    else cand[0].assign(blocks_mixed, blocks_mixed + 4);
    if (run->refill_period > 0) cand[1] = {run->refill_period};
    else if (fp64) cand[1].assign(ks_fp64, ks_fp64 + 4);
    else cand[1].assign(ks_mixed, ks_mixed + 4);
    if (run->flights_per_phase > 0) cand[2] = {run->flights_per_phase};
    else if (fp64) cand[2].assign(ms_fp64, ms_fp64 + 1);
    else cand[2].assign(ms_mixed, ms_mixed + 4);
    // start: a middle shape (one flight per phase with the banded majorant,
    // whose flights are mostly real; four with the global one)
    auto pick = [](const std::vector<int> &c, int want) {
        for (int v : c)
            if (v == want) return v;
        return c[c.size() / 2];
    };
    int cur[3] = {pick(cand[0], fp64 ? 256 : 896), pick(cand[1], 16),
                  pick(cand[2], r.majorant == GT_MAJORANT_BANDED ? 1 : 4)};
    gt_stats st{};
    r.block = cur[0];
    r.refill_period = cur[1];
    r.flights_per_phase = cur[2];
    int rc = avalanche_run(ctx, &r, out, ws, ws_bytes, stream, &st);  // warm-up
    if (rc != GT_OK) return rc;
    // measured shapes, so that no shape runs twice
    std::vector<gt_tune_point> seen;
    int n = 0;
    auto measure = [&](int b, int k, int m) -> double {
        for (const gt_tune_point &q : seen)
            if (q.block == b && q.refill_period == k && q.flights_per_phase == m)
                return q.real_per_ms;
        r.block = b;
        r.refill_period = k;
        r.flights_per_phase = m;
        gt_tune_point pt{b, k, m, 0, 0.0, 0.0};
        if (avalanche_run(ctx, &r, out, ws, ws_bytes, stream, &st) == GT_OK) {
            pt.transport_ms = st.transport_ms;
            pt.real_per_ms =
                st.transport_ms > 0 ? (double)st.real_collisions / st.transport_ms : 0.0;
        }
        seen.push_back(pt);
        if (points && n < max_points) points[n] = pt;
        ++n;
        return pt.real_per_ms;
    };
    // coordinate descent: each dimension in turn takes its best value with
    // the others held, until a whole sweep changes nothing (at most 4)
    double top = measure(cur[0], cur[1], cur[2]);
    for (int sweep = 0; sweep < 4; ++sweep) {
        bool changed = false;
        for (int d = 0; d < 3; ++d) {
            for (int v : cand[d]) {
                int s3[3] = {cur[0], cur[1], cur[2]};
                s3[d] = v;
                const double x = measure(s3[0], s3[1], s3[2]);
                if (x > top) {
                    top = x;
                    changed = changed || v != cur[d];
                    cur[d] = v;
                }
            }
        }
        if (!changed) break;
    }
    if (n_points) *n_points = n;
    if (!(top > 0.0)) return GT_ERR_UNSUPPORTED;
    const int pi = fp64 ? 0 : 1, mi = r.majorant == GT_MAJORANT_BANDED ? 1 : 0;
    const int vi = run_variant(ctx, &r);
    ctx->tuned_block[pi][ctx->field.kind][mi][vi] = cur[0];
    ctx->tuned_k[pi][ctx->field.kind][mi][vi] = cur[1];
    ctx->tuned_m[pi][ctx->field.kind][mi][vi] = cur[2];
    for (const gt_tune_point &q : seen)
        if (q.block == cur[0] && q.refill_period == cur[1] && q.flights_per_phase == cur[2])
            *best = q;
    return GT_OK;
}

int avalanche_observables(gt_ctx *ctx, const gt_endpoints *ep, int64_t n_endpoints,
                          int32_t n_avalanches, const int32_t *n_prim, int32_t collect_status,
                          int32_t drift_status, double gap, double *obs, void *stream)
{
    if (!ctx || !ep || !obs || n_endpoints < 0 || n_avalanches < 0 || n_endpoints > ep->capacity)
        return GT_ERR_ARG;
    if (n_avalanches > 0 && !n_prim) return GT_ERR_ARG;
    if (n_endpoints > 0 && (!ep->x0 || !ep->y0 || !ep->z0 || !ep->t0 || !ep->x1 || !ep->y1 ||
                            !ep->z1 || !ep->t1 || !ep->status || !ep->aval))
        return GT_ERR_ARG;
    DeviceGuard dg(ctx->device);
    if (!dg.ok) return GT_ERR_CUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t need_counts = (size_t)std::max(n_avalanches, 1);
    long long nb = (n_endpoints + 255) / 256;
    nb = std::max(1LL, std::min<long long>(nb, (long long)ctx->sms * 4));
    if (ctx->obs_counts_cap < need_counts) {
        if (ctx->d_obs_counts) cudaFree(ctx->d_obs_counts);
        ctx->d_obs_counts = nullptr;
        ctx->obs_counts_cap = 0;
        GT_CUDA(ctx, cudaMalloc((void **)&ctx->d_obs_counts, sizeof(unsigned long long) * need_counts));
        ctx->obs_counts_cap = need_counts;
    }
    if (ctx->obs_partials_cap < (size_t)nb * 5) {
        if (ctx->d_obs_partials) cudaFree(ctx->d_obs_partials);
        ctx->d_obs_partials = nullptr;
        ctx->obs_partials_cap = 0;
        GT_CUDA(ctx, cudaMalloc((void **)&ctx->d_obs_partials, sizeof(double) * (size_t)nb * 5));
        ctx->obs_partials_cap = (size_t)nb * 5;
    }
    RunParams p{};
    p.x0 = ep->x0; p.y0 = ep->y0; p.z0 = ep->z0; p.t0 = ep->t0;
    p.x1 = ep->x1; p.y1 = ep->y1; p.z1 = ep->z1; p.t1 = ep->t1;
    p.status = ep->status; p.aval = ep->aval;
    p.n_avalanches = n_avalanches;
    GT_CUDA(ctx, launch_observables(p, n_endpoints, n_avalanches, n_prim, collect_status,
                                    drift_status, gap, ctx->d_obs_counts, ctx->d_obs_partials,
                                    (int)nb, obs, s));
    GT_CUDA(ctx, cudaStreamSynchronize(s));
    return GT_OK;
}

}  // extern "C"
