// gt_kernels.cuh -- transport kernels (templates), instantiated per precision
// in gt_kernels_fp64.cu and gt_kernels_mixed.cu.
//
//   k_batched          one persistent launch for every avalanche: each lane
//                      holds one electron for a round of K flights; lanes
//                      without an electron take tickets on a global queue
//                      (warp ballot + prefix sum, one atomic per warp);
//                      ionisation appends the new electron to the queue the
//                      same way; the launch ends when every queued electron
//                      has finished (done == tail), or on a bounded wait.
//   k_plain_transport  one generation of one avalanche: every active electron
//                      flies until it ionises or finishes (Fig. 2 "electron
//                      transport"); a separate compaction launch then removes
//                      finished electrons and appends the new ones ("stack
//                      processing"), and the host loops until none is left.
#pragma once

#include "gt_device.cuh"

namespace gt {

constexpr unsigned FULL = 0xFFFFFFFFu;

// Builds of the batched kernel's collision round (its template parameter MP).
constexpr int kRoundAny = 0;       // flights per round from the run (flights_per_phase)
constexpr int kRoundOne = 1;       // one flight per round
constexpr int kRoundCommon = 2;    // one flight per round, the step built for the common run
constexpr int kRoundCrossing = 3;  // the same with exact crossings alone
constexpr int kRoundSignal = 4;    // the same with induced signals alone

// Row stride of the FP32 table staged in shared memory: odd, so that the
// rows of a warp's random energies start on all 32 banks.
__host__ __device__ inline int smem_stride(int n_levels) { return n_levels | 1; }

// Dynamic shared memory: the per-thread FP64 position/time bases
// [4][blockDim] (mixed precision), the per-thread collision tallies
// [L][blockDim], the banded-majorant range-max table, and (optionally) the
// FP32 cumulative table with an odd row stride.
__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

__host__ __device__ inline size_t shared_bytes(int n_levels, int n_nodes, int block, bool table,
                                               int band_entries)
{
    size_t b = (size_t)4 * block * sizeof(double);
    b += align16((size_t)n_levels * block * sizeof(uint32_t));
    b += align16((size_t)band_entries * sizeof(float));
    if (table) b += (size_t)smem_stride(n_levels) * n_nodes * sizeof(float);
    return b;
}

// Per-CTA statistics and per-warp wait bookkeeping (static shared memory).
struct BlockState {
    unsigned long long flights, real, nul;
    unsigned long long last_done[32], last_tail[32], t_progress[32];
    unsigned int sleep_ns[32];
    unsigned long long t_start;  // %globaltimer at the start of the run
};

template <bool SMEM_TABLE>
__device__ __forceinline__ Tables stage_tables(const RunParams &p, unsigned char *smem,
                                               BlockState &bs)
{
    __shared__ double s_thr[GT_MAX_LEVELS];
    __shared__ float s_thr_f[GT_MAX_LEVELS];
    __shared__ float s_xi0_f[GT_MAX_LEVELS];
    __shared__ float s_screen_f[GT_MAX_LEVELS];
    __shared__ int s_type[GT_MAX_LEVELS];
    const int L = p.gas.n_levels;
    double *s_base = reinterpret_cast<double *>(smem);
    const size_t off_tally = (size_t)4 * blockDim.x * sizeof(double);
    uint32_t *s_tally = reinterpret_cast<uint32_t *>(smem + off_tally);
    const int nb = p.gas.n_bands * p.gas.band_levels;
    const size_t off_band = off_tally + align16((size_t)L * blockDim.x * sizeof(uint32_t));
    float *s_band = reinterpret_cast<float *>(smem + off_band);
    float *s_cum = reinterpret_cast<float *>(smem + off_band + align16((size_t)nb * sizeof(float)));
    for (int i = threadIdx.x; i < nb; i += blockDim.x) s_band[i] = p.gas.band32[i];
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        s_thr[i] = p.gas.thr[i];
        s_thr_f[i] = (float)p.gas.thr[i];
        s_xi0_f[i] = (float)p.gas.xi0[i];
        s_screen_f[i] = (float)p.gas.screen[i];
        s_type[i] = p.gas.type[i];
    }
    for (int i = threadIdx.x; i < L * (int)blockDim.x; i += blockDim.x) s_tally[i] = 0u;
    const int S = smem_stride(L);
    if (SMEM_TABLE) {
        const int N = p.gas.n_nodes;
        for (int i = threadIdx.x; i < N * L; i += blockDim.x) {
            const int k = i / L, j = i - k * L;
            s_cum[k * S + j] = p.gas.cum32[i];
        }
    }
    if (threadIdx.x == 0) {
        bs.flights = bs.real = bs.nul = 0ull;
        bs.t_start = p.hdr->t_start;
    }
    if (threadIdx.x < 32) {
        bs.last_done[threadIdx.x] = ~0ull;
        bs.last_tail[threadIdx.x] = ~0ull;
        bs.t_progress[threadIdx.x] = 0ull;
        bs.sleep_ns[threadIdx.x] = 64u;
    }
    __syncthreads();
    Tables tb;
    tb.band32 = s_band;
    tb.cum32 = SMEM_TABLE ? s_cum : p.gas.cum32;
    tb.stride32 = SMEM_TABLE ? S : L;
    tb.cum64 = p.gas.cum64;
    tb.type = s_type;
    tb.thr = s_thr;
    tb.thr_f = s_thr_f;
    tb.xi0_f = s_xi0_f;
    tb.screen_f = s_screen_f;
    tb.tally = s_tally;
    tb.base = s_base;
    return tb;
}

// Block statistics to the run header (after the block's last transport).
__device__ __forceinline__ void flush_block_stats(const RunParams &p, BlockState &bs)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(&p.hdr->flights, bs.flights);
        atomicAdd(&p.hdr->real, bs.real);
        atomicAdd(&p.hdr->nul, bs.nul);
    }
}

// Move an electron's per-level collision counts from shared memory to the
// avalanche's tallies; returns the number of real collisions moved.
__device__ __forceinline__ unsigned long long flush_tally(const RunParams &p, const Tables &tb,
                                                          int aval, uint32_t nnull,
                                                          uint32_t n0 = 0u)
{
    const int L = p.gas.n_levels;
    uint64_t *tal = p.tallies + (int64_t)aval * (L + 1);
    unsigned long long real = 0;
    // level 0's collisions counted in a register (the straight-line path)
    tb.tally[threadIdx.x] += n0;
    for (int j = 0; j < L; ++j) {
        uint32_t &c = tb.tally[j * blockDim.x + threadIdx.x];
        if (c) {
            atomicAdd(reinterpret_cast<unsigned long long *>(tal + j), (unsigned long long)c);
            real += c;
            c = 0u;
        }
    }
    if (nnull) atomicAdd(reinterpret_cast<unsigned long long *>(tal + L), (unsigned long long)nnull);
    return real;
}

// An electron has finished: write its endpoint and move its counts.
template <bool GEO, class E>
__device__ __forceinline__ void finish(const RunParams &p, const Tables &tb, const E &e,
                                       BlockState &bs)
{
    if (GEO) e.signal_end(p);  // induced signals are built only into GEO kernels
    e.write_end(p);
    const unsigned long long real = flush_tally(p, tb, e.aval, e.nnull, e.level0_count());
    atomicAdd(&bs.flights, (unsigned long long)e.nf);
    atomicAdd(&bs.real, real);
    atomicAdd(&bs.nul, (unsigned long long)e.nnull);
}

// Warp-collective append of the lanes' new electrons to the queue: ballot,
// one atomic on the tail per warp, each lane's slot = base + its rank.
// Returns the number of this lane's electrons dropped for lack of capacity
// (they count as finished so that the queue can drain).
template <class E>
__device__ __forceinline__ int push_children(const RunParams &p, bool want, const E &parent,
                                             const typename E::ChildT &ch, int lane)
{
    bool ok = want;
    if (want && p.size_limit) {
        const unsigned long long old = atomicAdd(p.created + parent.aval, 1ull);
        if (old >= p.size_limit) {
            ok = false;
            atomicAdd(&p.hdr->dropped, 1ull);
        }
    }
    const unsigned m = __ballot_sync(FULL, ok);
    if (!m) return 0;
    const int leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(&p.hdr->tail, (unsigned long long)__popc(m));
    base = __shfl_sync(FULL, base, leader);
    if (!ok) return 0;
    const unsigned long long s = base + __popc(m & lanemask_lt());
    if (s >= (unsigned long long)p.capacity) {
        atomicAdd(&p.hdr->dropped, 1ull);
        atomicOr(&p.hdr->error, ERR_OVERFLOW);
        return 1;
    }
    store_birth(p, (int64_t)s, parent, ch);
    // the release store orders the record's stores before the flag
    st_release_u32(p.ready + s, 1u);
    return 0;
}

template <class E, int FK, bool SMEM_TABLE, int MAXT, int MP = 0, bool PHYS = true,
          bool GEO = true>
__global__ void __launch_bounds__(MAXT) k_batched(const RunParams p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ BlockState bs;
    const Tables tb = stage_tables<SMEM_TABLE>(p, smem, bs);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int K = p.refill_period;

    E e;
    e.bind(tb);
    bool has = false;
    long long ticket = -1;

    // a run whose arguments failed the device checks stops at once
    unsigned err0 = 0;
    if (lane == 0) err0 = *reinterpret_cast<volatile unsigned *>(&p.hdr->error);
    const bool stop0 = (__shfl_sync(FULL, err0, 0) & (ERR_TIMEOUT | ERR_BADARG)) != 0;

    // tickets requested at the end of the previous iteration (the atomic's
    // round trip overlaps that iteration's endpoint writes and flushes); in
    // the common-run builds without sub-steps, crossings or signals, whose
    // registers have room for it
    constexpr bool kPrefetch = MP == kRoundCommon && !GEO;
    unsigned pre_m = 0u;
    unsigned long long pre_base = 0ull;
    for (; !stop0;) {
        if (kPrefetch && pre_m) {
            const int leader = __ffs(pre_m) - 1;
            const unsigned long long base = __shfl_sync(FULL, pre_base, leader);
            if ((pre_m >> lane) & 1u) ticket = (long long)(base + __popc(pre_m & lanemask_lt()));
            pre_m = 0u;
        }
        // lanes without an electron take queue tickets: one atomic per warp
        const bool need = !has && ticket < 0;
        const unsigned m = __ballot_sync(FULL, need);
        if (m) {
            const int leader = __ffs(m) - 1;
            unsigned long long base = 0;
            if (lane == leader) base = atomicAdd(&p.hdr->head, (unsigned long long)__popc(m));
            base = __shfl_sync(FULL, base, leader);
            if (need) ticket = (long long)(base + __popc(m & lanemask_lt()));
        }
        int retired = 0;
        if (!has && ticket >= 0 && ticket < p.capacity) {
            if (ld_acquire_u32(p.ready + ticket)) {
                e.template load_birth<FK, GEO>(p, ticket);
                ticket = -1;
                has = true;
                if (e.template check_start<FK>(p) & EV_RETIRE) {
                    finish<GEO>(p, tb, e, bs);
                    has = false;
                    retired = 1;
                }
            }
        }

        if (!__any_sync(FULL, has)) {
            // the whole warp waits: finished when every queued electron is done
            const int r = __reduce_add_sync(FULL, retired);
            if (r) {
                if (lane == 0) atomicAdd(&p.hdr->done, (unsigned long long)r);
                continue;
            }
            int verdict = 0;  // 0 wait, 1 finished, 2 give up
            if (lane == 0) {
                const unsigned long long d = ld_acquire_u64(&p.hdr->done);
                const unsigned long long tl = ld_acquire_u64(&p.hdr->tail);
                const unsigned err = *reinterpret_cast<volatile unsigned *>(&p.hdr->error);
                const unsigned long long now = globaltimer();
                if (d == tl) {
                    verdict = 1;
                } else if (err & (ERR_TIMEOUT | ERR_BADARG)) {
                    verdict = 2;
                } else if (d != bs.last_done[wid] || tl != bs.last_tail[wid]) {
                    bs.last_done[wid] = d;
                    bs.last_tail[wid] = tl;
                    bs.t_progress[wid] = now;
                    bs.sleep_ns[wid] = 64u;
                } else if ((long long)(now - bs.t_progress[wid]) > p.spin_limit_ns ||
                           (long long)(now - bs.t_start) > p.time_limit_ns) {
                    atomicOr(&p.hdr->error, ERR_TIMEOUT);
                    verdict = 2;
                }
                if (!verdict) {
                    __nanosleep(bs.sleep_ns[wid]);
                    bs.sleep_ns[wid] = bs.sleep_ns[wid] < 8192u ? bs.sleep_ns[wid] * 2u : 8192u;
                }
            }
            if (__shfl_sync(FULL, verdict, 0)) break;
            continue;
        }

        if constexpr (E::kTwoPhase) {
            // K collision rounds between refills.  In each, lanes without a
            // pending collision fly (at most M flights) until they meet a
            // real one; then the warp applies its lanes' collisions together.
            // kRoundOne builds the one-flight round (M = 1) at compile time;
            // kRoundCommon, kRoundCrossing and kRoundSignal do too, with the
            // step built for the common run (MixedElectron::advance with
            // MAJ = 1), and with exact crossings / induced signals alone
            // (MAJ = 2 / 3)
            constexpr int MPF = MP >= kRoundCommon ? 1 : MP;
            constexpr int MAJ = MP >= kRoundCommon ? MP - kRoundOne : 0;
            const int M = MPF ? MPF : p.flights_per_phase;
            // an electron that finishes during the rounds keeps its lane (a
            // lane takes a new electron only at the next refill) and is
            // written out after the last round, together with the warp's
            // other finished electrons, instead of one divergent pass each
            bool fin = false;
            for (int k = 0; k < K; ++k) {
                typename E::Pending pd;
                pd.real = false;
                for (int mm = 0; mm < M; ++mm) {
                    const bool go = has && !pd.real;
                    if (MPF != 1 && !__any_sync(FULL, go)) break;
                    if (go && (e.template advance<FK, GEO, MAJ>(p, tb, pd) & EV_RETIRE)) {
                        has = false;
                        fin = true;
                    }
                }
                typename E::ChildT ch;
                int ev = EV_NONE;
                if (pd.real) ev = e.template collide<FK, PHYS, MAJ>(p, tb, pd, ch);
                if (__any_sync(FULL, ev & EV_CHILD))
                    retired += push_children(p, (ev & EV_CHILD) != 0, e, ch, lane);
                if (ev & EV_RETIRE) {
                    has = false;
                    fin = true;
                }
            }
            // the lanes that will need an electron ask for tickets now
            if constexpr (kPrefetch) {
                pre_m = __ballot_sync(FULL, !has && ticket < 0);
                if (pre_m && lane == __ffs(pre_m) - 1)
                    pre_base = atomicAdd(&p.hdr->head, (unsigned long long)__popc(pre_m));
            }
            if (fin) {
                finish<GEO>(p, tb, e, bs);
                ++retired;
            }
        } else {
            // K flights per electron between refills
            for (int k = 0; k < K; ++k) {
                typename E::ChildT ch;
                int ev = EV_NONE;
                if (has) ev = e.template fly<FK>(p, tb, ch);
                if (__any_sync(FULL, ev & EV_CHILD))
                    retired += push_children(p, (ev & EV_CHILD) != 0, e, ch, lane);
                if (ev & EV_RETIRE) {
                    finish<GEO>(p, tb, e, bs);
                    has = false;
                    ++retired;
                }
            }
        }
        if (has) e.template round_end<FK>(p);

        // finished electrons are counted; the count only decides when the
        // launch may end (done == tail), and no kernel reads an endpoint, so
        // no fence orders the endpoint writes before it (the launch's end
        // makes them visible to the host)
        const int r = __reduce_add_sync(FULL, retired);
        if (r && lane == 0) atomicAdd(&p.hdr->done, (unsigned long long)r);
        // the run-wide checks: the time budget, and an abort from any warp
        unsigned stop = 0;
        if (lane == 0) {
            const unsigned err = *reinterpret_cast<volatile unsigned *>(&p.hdr->error);
            if ((long long)(globaltimer() - bs.t_start) > p.time_limit_ns) {
                atomicOr(&p.hdr->error, ERR_TIMEOUT);
                stop = 1u;
            }
            stop |= err & (ERR_TIMEOUT | ERR_BADARG);
        }
        if (__shfl_sync(FULL, stop, 0)) break;
    }
    flush_block_stats(p, bs);
}

// One generation of one avalanche (plain mode): every electron of `cur`
// flies until it ionises (it stays alive and its new electron goes to
// `fresh`) or finishes (alive = 0).
template <class E, int FK, bool SMEM_TABLE, int MAXT, bool PHYS = true, bool GEO = true>
__global__ void __launch_bounds__(MAXT)
    k_plain_transport(const RunParams p, const Stack cur, long long n_active, const Stack fresh,
                      int parity, int aval)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ BlockState bs;
    const Tables tb = stage_tables<SMEM_TABLE>(p, smem, bs);
    if (blockIdx.x == 0 && threadIdx.x == 0) p.hdr->n_next[parity] = 0ull;
    const unsigned long long t_start = p.hdr->t_start;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_active) return;

    E e;
    e.bind(tb);
    e.template restore<FK, GEO>(p, cur, i, aval);
    const uint32_t nf0 = e.nf, nr0 = e.nreal;
    typename E::ChildT ch;
    int ev = EV_NONE;
    if (e.nf == 0u) ev = e.template check_start<FK>(p);
    unsigned long long k = 0;
    while (ev == EV_NONE) {
        ev = e.template fly<FK, PHYS, GEO>(p, tb, ch);
        if ((++k & 4095ull) == 0ull) {
            if ((long long)(globaltimer() - t_start) > p.time_limit_ns) {
                atomicOr(&p.hdr->error, ERR_TIMEOUT);
                break;
            }
        }
    }
    if (ev & EV_CHILD) {
        const unsigned long long s = atomicAdd(&p.hdr->tail, 1ull);
        if (s < (unsigned long long)p.capacity) {
            store_birth(p, (int64_t)s, e, ch);
            p.ready[s] = 1u;
            const unsigned long long j = atomicAdd(&p.hdr->n_new[parity], 1ull);
            e.position(p, fresh.x[j], fresh.y[j], fresh.z[j], fresh.t[j]);
            fresh.vx[j] = (double)ch.vx; fresh.vy[j] = (double)ch.vy; fresh.vz[j] = (double)ch.vz;
            fresh.nf[j] = 0u; fresh.nreal[j] = 0u; fresh.uid[j] = ch.uid;
            fresh.slot[j] = (int64_t)s;
        } else {
            atomicAdd(&p.hdr->dropped, 1ull);
            atomicOr(&p.hdr->error, ERR_OVERFLOW);
        }
    }
    // per-level counts of this stretch go to the avalanche's tallies
    flush_tally(p, tb, aval, e.nnull, e.level0_count());
    atomicAdd(&p.hdr->flights, (unsigned long long)(e.nf - nf0));
    atomicAdd(&p.hdr->real, (unsigned long long)(e.nreal - nr0));
    atomicAdd(&p.hdr->nul, (unsigned long long)e.nnull);
    if (ev & EV_RETIRE) {
        if (GEO) e.signal_end(p);
        e.write_end(p);
        cur.alive[i] = 0;
    } else {
        e.template save<FK, GEO>(p, cur, i);
        cur.alive[i] = 1;
    }
}

}  // namespace gt
