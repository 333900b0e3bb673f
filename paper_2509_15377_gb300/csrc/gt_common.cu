// gt_common.cu -- precision-independent kernels: queue seeding (primary
// injection), plain-mode stack set-up and compaction ("stack processing",
// Sec. 2), per-avalanche electron counts and the observables reduction.
#include "gt_kernels.cuh"
#include "gt_launch.h"

#include <cstring>

namespace gt {

// Primary injection: primary i goes to queue / endpoint slot i with its
// start record, birth velocity sqrt(2 a e) * direction and a filled flag.
__global__ void k_seed(const RunParams p, const SeedArgs a)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i0 == 0) {  // the header was zeroed before this launch
        Header *h = p.hdr;
        h->tail = (unsigned long long)a.n + (a.unfilled_slot ? 1ull : 0ull);
        h->t_start = globaltimer();
    }
    for (long long i = i0; i < a.n; i += stride) {
        int av = a.aval[i];
        if (av < 0 || av >= p.n_avalanches || !(a.e[i] >= 0.0)) {
            // an invalid primary is flagged; the run is abandoned before transport
            atomicOr(&p.hdr->error, ERR_BADARG);
            av = 0;
        }
        const double s = sqrt(kTwoAccel * fmax(a.e[i], 0.0));
        p.x0[i] = a.x[i]; p.y0[i] = a.y[i]; p.z0[i] = a.z[i]; p.t0[i] = a.t[i]; p.e0[i] = a.e[i];
        p.bvx[i] = s * a.dx[i]; p.bvy[i] = s * a.dy[i]; p.bvz[i] = s * a.dz[i];
        p.belem[i] = -1;
        p.uid[i] = a.uid[i];
        p.aval[i] = av;
        p.status[i] = 0;
        p.ready[i] = 1u;
        if (p.size_limit) atomicAdd(p.created + av, 1ull);
    }
}

cudaError_t launch_seed(const RunParams &p, const SeedArgs &a, cudaStream_t s)
{
    long long blocks = (a.n + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (blocks > 4096) blocks = 4096;
    k_seed<<<(unsigned)blocks, 256, 0, s>>>(p, a);
    return cudaGetLastError();
}

// Plain mode: the first generation of one avalanche from its primaries' slots.
__global__ void k_plain_init(const RunParams p, const Stack st, const long long *order,
                             long long first, long long count)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const long long s = order[first + i];
    st.x[i] = p.x0[s]; st.y[i] = p.y0[s]; st.z[i] = p.z0[s]; st.t[i] = p.t0[s];
    st.vx[i] = p.bvx[s]; st.vy[i] = p.bvy[s]; st.vz[i] = p.bvz[s];
    st.nf[i] = 0u; st.nreal[i] = 0u;
    st.uid[i] = p.uid[s];
    st.slot[i] = s;
}

cudaError_t launch_plain_init(const RunParams &p, const Stack &st, const long long *order,
                              long long first, long long count, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    k_plain_init<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(p, st, order, first, count);
    return cudaGetLastError();
}

// Stack processing: still-active electrons of `cur` followed by the new
// ones of `fresh`, compacted into `next` (warp ballot, block prefix sum,
// one atomic per block for the block's base).
__global__ void k_plain_compact(const RunParams p, const PlainArgs a)
{
    __shared__ int warp_count[32];
    __shared__ unsigned long long block_base;
    const unsigned long long n_new = p.hdr->n_new[a.parity];
    const long long n_cur = a.n_active;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    bool keep = false;
    const Stack *src = &a.cur;
    long long j = i;
    if (i < n_cur) {
        keep = a.cur.alive[i] != 0;
    } else if (i - n_cur < (long long)n_new) {
        keep = true;
        src = &a.fresh;
        j = i - n_cur;
    }
    const unsigned m = __ballot_sync(FULL, keep);
    if (lane == 0) warp_count[wid] = __popc(m);
    __syncthreads();
    if (threadIdx.x == 0) {
        int total = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            const int c = warp_count[w];
            warp_count[w] = total;
            total += c;
        }
        block_base = total ? atomicAdd(&p.hdr->n_next[a.parity], (unsigned long long)total) : 0ull;
        if (blockIdx.x == 0) p.hdr->n_new[a.parity ^ 1] = 0ull;
    }
    __syncthreads();
    if (!keep) return;
    const long long d = (long long)block_base + warp_count[wid] + __popc(m & lanemask_lt());
    const Stack &S = *src;
    a.next.x[d] = S.x[j]; a.next.y[d] = S.y[j]; a.next.z[d] = S.z[j]; a.next.t[d] = S.t[j];
    a.next.vx[d] = S.vx[j]; a.next.vy[d] = S.vy[j]; a.next.vz[d] = S.vz[j];
    a.next.nf[d] = S.nf[j]; a.next.nreal[d] = S.nreal[j];
    a.next.uid[d] = S.uid[j]; a.next.slot[d] = S.slot[j];
}

cudaError_t launch_plain_compact(const RunParams &p, const PlainArgs &a, cudaStream_t s)
{
    // every electron ionises at most once per generation: at most 2 n entries
    const long long n = 2 * a.n_active;
    if (n <= 0) return cudaSuccess;
    k_plain_compact<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, a);
    return cudaGetLastError();
}

// Electrons stored per avalanche (filled slots of the queue).
__global__ void k_count_electrons(const RunParams p)
{
    unsigned long long n = p.hdr->tail;
    if (n > (unsigned long long)p.capacity) n = (unsigned long long)p.capacity;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += stride) {
        if (p.ready[i])
            atomicAdd(reinterpret_cast<unsigned long long *>(p.electrons + p.aval[i]), 1ull);
    }
}

cudaError_t launch_count_electrons(const RunParams &p, int sms, cudaStream_t s)
{
    k_count_electrons<<<sms * 4, 256, 0, s>>>(p);
    return cudaGetLastError();
}

// Largest |E| over the nodes of a grid map (bits of non-negative floats
// order like the floats, so an integer atomicMax finds the largest).
__global__ void k_grid_emax(const float4 *grid, long long n, unsigned *out)
{
    float m = 0.0f;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float4 e = __ldg(grid + i);
        m = fmaxf(m, sqrtf(e.x * e.x + e.y * e.y + e.z * e.z));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(FULL, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

cudaError_t grid_emax(const float4 *grid, long long n, int sms, double *emax)
{
    unsigned *d = nullptr, h = 0;
    cudaError_t e = cudaMalloc((void **)&d, sizeof(unsigned));
    if (e != cudaSuccess) return e;
    e = cudaMemset(d, 0, sizeof(unsigned));
    if (e == cudaSuccess) {
        k_grid_emax<<<sms * 4, 256>>>(grid, n, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(unsigned), cudaMemcpyDeviceToHost);
    cudaFree(d);
    float f;
    memcpy(&f, &h, sizeof(f));
    // one ulp up: the FP32 norm above may round below the exact one
    *emax = (double)f * (1.0 + 1e-6);
    return e;
}

// ---------------------------------------------------------- observables
constexpr int OBS_BLOCK = 256;

__device__ __forceinline__ double block_sum(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    return t;  // valid in thread 0
}

// Pass 1: per-avalanche count of electrons ending with collect_status and
// per-block FP64 sums of dz, dt, dx^2 + dy^2, dz^2 and the electron count
// over electrons ending with drift_status (any finished one if < 0).
__global__ void k_obs_pass1(const RunParams p, long long n, int collect_status, int drift_status,
                            unsigned long long *counts, double *partials)
{
    __shared__ double sh[32];
    double s_dz = 0, s_dt = 0, s_tr = 0, s_dz2 = 0, s_n = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int st = p.status[i];
        if (st == 0) continue;
        const int av = p.aval[i];
        if (st == collect_status && av >= 0 && av < p.n_avalanches) atomicAdd(counts + av, 1ull);
        if (drift_status < 0 || st == drift_status) {
            const double dx = p.x1[i] - p.x0[i], dy = p.y1[i] - p.y0[i];
            const double dz = p.z1[i] - p.z0[i], dt = p.t1[i] - p.t0[i];
            s_dz += dz; s_dt += dt; s_tr += dx * dx + dy * dy; s_dz2 += dz * dz; s_n += 1.0;
        }
    }
    const double v[5] = {s_dz, s_dt, s_tr, s_dz2, s_n};
    for (int k = 0; k < 5; ++k) {
        const double t = block_sum(v[k], sh);
        if (threadIdx.x == 0) partials[(long long)blockIdx.x * 5 + k] = t;
    }
}

// Pass 2 (one block): gain statistics over avalanches with primaries and the
// transport observables from the block partials, in a fixed order.
__global__ void k_obs_pass2(int n_aval, const int32_t *n_prim, const unsigned long long *counts,
                            const double *partials, int n_blocks, double gap, double *obs)
{
    __shared__ double sh[32];
    double g = 0, g2 = 0, na = 0;
    for (int a = threadIdx.x; a < n_aval; a += blockDim.x) {
        if (n_prim[a] > 0) {
            const double x = (double)counts[a] / (double)n_prim[a];
            g += x; g2 += x * x; na += 1.0;
        }
    }
    const double G = block_sum(g, sh), G2 = block_sum(g2, sh), NA = block_sum(na, sh);
    if (threadIdx.x != 0) return;
    double s[5] = {0, 0, 0, 0, 0};
    for (int b = 0; b < n_blocks; ++b)
        for (int k = 0; k < 5; ++k) s[k] += partials[(long long)b * 5 + k];
    const double mean = NA > 0 ? G / NA : 0.0;
    const double var = NA > 1 ? (G2 - NA * mean * mean) / (NA - 1.0) : 0.0;
    obs[0] = mean;
    obs[1] = NA > 0 ? sqrt(fmax(var, 0.0) / NA) : 0.0;
    obs[2] = NA;
    const double n = s[4];
    obs[3] = s[1] != 0.0 ? s[0] / s[1] : 0.0;
    const double mt = n > 0 ? s[1] / n : 0.0;
    obs[4] = (n > 0 && mt > 0) ? (s[2] / n) / (4.0 * mt) : 0.0;
    const double mz = n > 0 ? s[0] / n : 0.0;
    obs[5] = (n > 1 && mt > 0) ? ((s[3] - n * mz * mz) / (n - 1.0)) / (2.0 * mt) : 0.0;
    obs[6] = n;
    obs[7] = (gap > 0 && mean > 0) ? log(mean) / gap : 0.0;
}

cudaError_t launch_observables(const RunParams &p, long long n_endpoints, int n_avalanches,
                               const int32_t *n_prim, int collect_status, int drift_status,
                               double gap, unsigned long long *scratch_counts,
                               double *scratch_partials, int n_blocks, double *obs,
                               cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(scratch_counts, 0,
                                    sizeof(unsigned long long) * (size_t)(n_avalanches > 0 ? n_avalanches : 1), s);
    if (e != cudaSuccess) return e;
    k_obs_pass1<<<n_blocks, OBS_BLOCK, 0, s>>>(p, n_endpoints, collect_status, drift_status,
                                               scratch_counts, scratch_partials);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    k_obs_pass2<<<1, 1024, 0, s>>>(n_avalanches, n_prim, scratch_counts, scratch_partials,
                                   n_blocks, gap, obs);
    return cudaGetLastError();
}

}  // namespace gt
