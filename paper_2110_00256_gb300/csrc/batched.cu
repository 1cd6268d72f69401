// batched.cu -- the substep over many patches (each with its own electrons,
// positrons and photons of uneven size) in four launches per step, whatever
// the number of patches: zero the firing counts, one evolution launch over all
// 3 x n segments, one event launch over all firing lists (photon emission of
// the leptons, pair production of the photons; with the learned sampler, one
// launch per process), one clamp.  The segment
// descriptors live in device memory owned by a qed_batch (made once), so the
// step allocates nothing and can be captured in a CUDA graph; with
// opts->d_step a captured step replays as many steps.  qed_tune_evolve picks
// the evolution launch shape (threads per CTA, CTAs per SM) by timing dry runs.
#include <cmath>
#include <cstring>
#include <vector>

#include "events.cuh"
#include "evolve_core.cuh"
#include "pipeline.cuh"
#include "pusher.cuh"

namespace qed {

qed_status check_opts(const qed_substep_opts *o);
template <typename T>
EventCommon<T> event_common(const qed_tables *t, int proc, uint64_t seed, int64_t step, const qed_substep_opts *o);

struct ClampEntry {
    unsigned long long *count;
    int64_t cap;
};

}  // namespace qed

struct qed_batch {
    int device;
    qed_precision prec;
    int n_patches;
    void *d_evolve;    // EvolveSeg<T>[3 n]: electrons, positrons, photons of patch 0, 1, ...
    void *d_qs;        // EventSeg<T>[2 n]: electrons -> photons, positrons -> photons
    void *d_bw;        // EventSeg<T>[n]: photons -> electrons, positrons
    int64_t **d_zero;  // [3 n] firing counts to zero
    qed::ClampEntry *d_clamp;  // [6 n] species and firing counts to clamp
    void *d_push;      // PushSeg<T>[3 n] when every species has positions, else NULL
    bool vec;
    bool push_vec;     // vec, and the positions 16-byte aligned too
    int64_t capacity_sum, fire_capacity_max;
    int threads, ctas_per_sm;  // tuned evolution launch shape (0: default)
};

namespace qed {

// one CTA of 256: zero the n firing counts; with stats, add the live counts of
// the species (the first three of every six clamp entries), clamped as the
// evolution clamps them, to QED_STAT_EVOLVED: the particles this step evolves,
// less the photons removed by pair production that are still in the arrays
// (QED_STAT_PAIRS - QED_STAT_COMPACTED: they are read, but not evolved)
__global__ void __launch_bounds__(256) zero_counts_kernel(int64_t *const *p, int n, const ClampEntry *e,
                                                          int n_patches, long long *stats)
{
    __shared__ long long s_sum[8];
    for (int i = threadIdx.x; i < n; i += blockDim.x) *p[i] = 0;
    if (!stats) return;
    long long live = 0;
    for (int i = threadIdx.x; i < 3 * n_patches; i += blockDim.x) {
        const ClampEntry &c = e[6 * (i / 3) + i % 3];
        const long long v = (long long)*c.count;  // as the evolution reads it
        live += v < 0 ? 0 : (v > c.cap ? c.cap : v);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) live += __shfl_xor_sync(0xffffffffu, live, o);
    if ((threadIdx.x & 31) == 0) s_sum[threadIdx.x >> 5] = live;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_sum[w];
        long long removed = stats[QED_STAT_PAIRS] - stats[QED_STAT_COMPACTED];
        removed = removed < 0 ? 0 : (removed > t ? t : removed);
        atomicAdd((unsigned long long *)(stats + QED_STAT_EVOLVED), (unsigned long long)(t - removed));
    }
}

__global__ void clamp_batch_kernel(const ClampEntry *e, int n, int64_t *step)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        unsigned long long *c = e[i].count;
        if (*c > (unsigned long long)e[i].cap) *c = e[i].cap;
    }
    if (step && blockIdx.x == 0 && threadIdx.x == 0) *step += 1;
}

// Block-wide prefix of the 32-entry chunk counts of n_seg firing lists into
// s_end (inclusive); s_n receives the clamped list lengths.  The lists are
// a[0 .. na) followed by b[0 .. n_seg - na).
template <typename T>
__device__ void chunk_prefix(const EventSeg<T> *a, int na, const EventSeg<T> *b, int n_seg, long long *s_end,
                             long long *s_n, long long *s_warp)
{
    const int per = (n_seg + blockDim.x - 1) / blockDim.x;
    const int s0 = threadIdx.x * per, s1 = min(n_seg, s0 + per);
    long long local = 0;
    for (int s = s0; s < s1; ++s) {
        const EventSeg<T> &g = s < na ? a[s] : b[s - na];
        const long long n = fire_n(g.fire_count, g.fire_cap);
        s_n[s] = n;
        local += (n + 31) / 32;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    long long acc = incl - local;
    for (int w = 0; w < warp; ++w) acc += s_warp[w];
    for (int s = s0; s < s1; ++s) {
        acc += (s_n[s] + 31) / 32;
        s_end[s] = acc;
    }
    __syncthreads();
}

__device__ __forceinline__ int find_seg(const long long *s_end, int n_seg, long long c)
{
    int lo = 0, hi = n_seg - 1;  // first s with s_end[s] > c
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (s_end[mid] > c)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

// dynamic shared memory: [InferSmem if MLP][s_end n][s_n n]
template <typename T, bool MLP, bool QS>
__global__ void __launch_bounds__(256, (MLP || sizeof(T) == 8) ? 1 : 4)
    event_batched_kernel(const EventSeg<T> *__restrict__ segs, int n_seg, const __grid_constant__ EventCommon<T> c)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ long long s_warp[8];
    InferSmem &S = *reinterpret_cast<InferSmem *>(smem_raw);
    long long *s_end = reinterpret_cast<long long *>(smem_raw + (MLP ? sizeof(InferSmem) : 0));
    long long *s_n = s_end + n_seg;
    if constexpr (MLP) mlp_stage(S.net, c.mlpv.w);
    chunk_prefix<T>(segs, n_seg, segs, n_seg, s_end, s_n, s_warp);
    const long long total = s_end[n_seg - 1];
    const int64_t step = event_step(c.d_step, c.step);
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarp = ((long long)gridDim.x * blockDim.x) >> 5;
    EventCounts k;
    for (long long ch = warp; ch < total; ch += nwarp) {
        const int s = find_seg(s_end, n_seg, ch);
        const int64_t base = (ch - (s ? s_end[s - 1] : 0)) * 32;
        if constexpr (QS)
            qs_event_chunk<T, MLP>(segs[s], c, step, base, s_n[s], S, k);
        else
            bw_event_chunk<T, MLP>(segs[s], c, step, base, s_n[s], S, k);
    }
    flush_counts(c.stats, k, QS);
}

// Both processes in one launch (table sampler): the photon emission of every
// lepton list and the pair production of every photon list touch disjoint
// particles (see events3_kernel), so their chunks run side by side.
// Dynamic shared memory: [s_end n][s_n n], n = n_qs + n_bw.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 1 : 4)
    event_batched_all_kernel(const EventSeg<T> *__restrict__ qs, int n_qs, const EventSeg<T> *__restrict__ bw,
                             int n_bw, const __grid_constant__ EventCommon<T> cq,
                             const __grid_constant__ EventCommon<T> cb)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ long long s_warp[8];
    InferSmem &S = *reinterpret_cast<InferSmem *>(smem_raw);  // (not touched without the learned sampler)
    const int n_seg = n_qs + n_bw;
    long long *s_end = reinterpret_cast<long long *>(smem_raw);
    long long *s_n = s_end + n_seg;
    chunk_prefix<T>(qs, n_qs, bw, n_seg, s_end, s_n, s_warp);
    const long long total = s_end[n_seg - 1];
    const int64_t step = event_step(cq.d_step, cq.step);
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarp = ((long long)gridDim.x * blockDim.x) >> 5;
    EventCounts kq, kb;
    for (long long ch = warp; ch < total; ch += nwarp) {
        const int s = find_seg(s_end, n_seg, ch);
        const int64_t base = (ch - (s ? s_end[s - 1] : 0)) * 32;
        if (s < n_qs)
            qs_event_chunk<T, false>(qs[s], cq, step, base, s_n[s], S, kq);
        else
            bw_event_chunk<T, false>(bw[s - n_qs], cb, step, base, s_n[s], S, kb);
    }
    flush_counts(cq.stats, kq, true);
    flush_counts(cb.stats, kb, false);
}

// ---------------------------------------------------------------------------
// The evolution over device-resident segments, FP32 with 16-byte-aligned
// arrays: the bulk-copy form of the single-call default.  The last warp of the
// CTA copies whole tiles (TP = CW x 32 x 4 particles of one segment) of the
// eleven streamed arrays into S shared-memory stages with cp.async.bulk; the CW
// consumer warps take four particles each, release the stage and evaluate them
// (the ragged last tile of a segment is read from global memory).  Tiles map
// to segments through the block-wide prefix of their tile counts.  Every wait
// is bounded (QED_STAT_WAIT_TIMEOUT counts a CTA that gave up).
// ---------------------------------------------------------------------------
constexpr int kSegArrays = 11;

__device__ __forceinline__ const float *seg_stream(const EvolveSeg<float> &g, int k)
{
    switch (k) {
    case 0: return g.px;
    case 1: return g.py;
    case 2: return g.pz;
    case 3: return g.ex;
    case 4: return g.ey;
    case 5: return g.ez;
    case 6: return g.bx;
    case 7: return g.by;
    case 8: return g.bz;
    case 9: return g.tau;
    default: return g.tau_c;
    }
}

__device__ __forceinline__ bool seg_wait(uint64_t *bar, uint32_t parity, volatile int *abort, long long limit)
{
    if (limit < kWaitCycles) {  // a caller's shorter limit: non-blocking probes (see evolve.cu)
        const long long t0 = clock64();
        while (!mbar_peek(bar, parity))
            if (*abort || clock64() - t0 > limit) return false;
        return true;
    }
    if (mbar_test(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_test(bar, parity)) {
        if (*abort || clock64() - t0 > limit) return false;
    }
    return true;
}

__device__ __forceinline__ void seg_give_up(int *abort, long long *stats)
{
    if (atomicExch(abort, 1) == 0) {
        note_error(QED_EW_WAIT_TIMEOUT);
        if (stats) atomicAdd((unsigned long long *)(stats + QED_STAT_WAIT_TIMEOUT), 1ull);
    }
}

template <int CW, int S>
__global__ void __launch_bounds__((CW + 1) * 32, 1)
    evolve_seg_bulk_kernel(const EvolveSeg<float> *__restrict__ segs, int n_seg, TablesView<float> tab, float dt,
                           float cut_qs, float cut_bw, long long *stats, int dry, long long wait_cycles)
{
    constexpr int THREADS = (CW + 1) * 32;
    constexpr int TP = CW * 32 * 4;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *s_stage = reinterpret_cast<float *>(smem_raw);  // [S][kSegArrays][TP]
    long long *s_end = reinterpret_cast<long long *>(smem_raw + (size_t)S * kSegArrays * TP * sizeof(float));
    long long *s_n = s_end + n_seg;
    __shared__ __align__(8) uint64_t s_full[S];
    __shared__ __align__(8) uint64_t s_empty[S];
    __shared__ float s_qs[QED_MAX_TABLE_N];
    __shared__ float s_bw[QED_MAX_TABLE_N];
    __shared__ long long s_warp[THREADS / 32];
    __shared__ int s_abort;

    for (int i = threadIdx.x; i < tab.qs_G.n; i += THREADS) s_qs[i] = tab.qs_G.ln_f[i];
    for (int i = threadIdx.x; i < tab.bw_T.n; i += THREADS) s_bw[i] = tab.bw_T.ln_f[i];
    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int k = 0; k < S; ++k) {
            mbar_init(&s_full[k], 1);
            mbar_init(&s_empty[k], CW);
        }
        mbar_fence_init();
    }
    const long long total = tile_prefix<float, THREADS>(segs, n_seg, TP, s_end, s_n, s_warp);  // ends with a barrier
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int *abort = &s_abort;
    // the producer/consumer hand-offs use the caller's limit; the final wait for
    // the copies in flight always the full one
    const long long limit = wait_cycles > 0 ? wait_cycles : kWaitCycles;

    if (warp == CW) {  // producer
        const uint64_t pol = l2_evict_first();
        int k = 0, s = 0;
        for (long long t = blockIdx.x; t < total; t += gridDim.x, ++k) {
            const int st = k % S;
            const uint32_t ph = (uint32_t)(k / S) & 1u;
            while (s_end[s] <= t) ++s;  // tiles ascend: the segment only moves forward
            const int64_t i0 = (t - (s ? s_end[s - 1] : 0)) * (int64_t)TP;
            if (!__all_sync(0xffffffffu, seg_wait(&s_empty[st], ph ^ 1u, abort, limit))) {
                if (lane == 0) seg_give_up(&s_abort, stats);
                break;
            }
            if (i0 + TP <= s_n[s]) {
                if (lane == 0) mbar_arrive_expect_tx(&s_full[st], kSegArrays * TP * (uint32_t)sizeof(float));
                __syncwarp();
                if (lane < kSegArrays)
                    bulk_g2s(s_stage + ((size_t)st * kSegArrays + lane) * TP, seg_stream(segs[s], lane) + i0,
                             TP * (uint32_t)sizeof(float), &s_full[st], pol);
            } else if (lane == 0) {
                mbar_arrive(&s_full[st]);
            }
        }
        for (int j = 1; j <= S && j <= k; ++j) {
            const int kk = k - j;
            if (!mbar_wait(&s_full[kk % S], (uint32_t)(kk / S) & 1u) && lane == 0) seg_give_up(&s_abort, stats);
        }
        return;
    }

    int bad = 0;
    int k = 0, s = 0;
    for (long long t = blockIdx.x; t < total; t += gridDim.x, ++k) {
        const int st = k % S;
        const uint32_t ph = (uint32_t)(k / S) & 1u;
        while (s_end[s] <= t) ++s;
        const EvolveSeg<float> &sg = segs[s];
        const int64_t n = s_n[s];
        const int64_t base = (t - (s ? s_end[s - 1] : 0)) * (int64_t)TP;
        const int64_t i0 = base + 4 * (int64_t)threadIdx.x;
        if (!__all_sync(0xffffffffu, seg_wait(&s_full[st], ph, abort, limit))) {
            if (lane == 0) seg_give_up(&s_abort, stats);
            break;
        }
        float px[4], py[4], pz[4], ex[4], ey[4], ez[4], bx[4], by[4], bz[4], tau[4], tc[4];
        bool full4;
        if (base + TP <= n) {
            const float4 *v = reinterpret_cast<const float4 *>(s_stage + (size_t)st * kSegArrays * TP) + threadIdx.x;
            constexpr int q = TP / 4;
            float4 w;
#define QED_UNPACK(arr, kk)                                \
    w = v[(kk) * q];                                       \
    arr[0] = w.x, arr[1] = w.y, arr[2] = w.z, arr[3] = w.w;
            QED_UNPACK(px, 0) QED_UNPACK(py, 1) QED_UNPACK(pz, 2);
            QED_UNPACK(ex, 3) QED_UNPACK(ey, 4) QED_UNPACK(ez, 5);
            QED_UNPACK(bx, 6) QED_UNPACK(by, 7) QED_UNPACK(bz, 8);
            QED_UNPACK(tau, 9) QED_UNPACK(tc, 10);
#undef QED_UNPACK
            full4 = true;
        } else {
            full4 = i0 + 4 <= n;
            if (full4) {
                load_vec<float, 4>(sg.px, i0, px);
                load_vec<float, 4>(sg.py, i0, py);
                load_vec<float, 4>(sg.pz, i0, pz);
                load_vec<float, 4>(sg.ex, i0, ex);
                load_vec<float, 4>(sg.ey, i0, ey);
                load_vec<float, 4>(sg.ez, i0, ez);
                load_vec<float, 4>(sg.bx, i0, bx);
                load_vec<float, 4>(sg.by, i0, by);
                load_vec<float, 4>(sg.bz, i0, bz);
                load_vec<float, 4>(sg.tau, i0, tau);
                load_vec<float, 4>(sg.tau_c, i0, tc);
            } else {
                load_scalar<float, 4>(sg, n, i0, px, py, pz, ex, ey, ez, bx, by, bz, tau, tc);
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&s_empty[st]);
        evolve_regs<float, 4>(sg, n, i0, full4, px, py, pz, ex, ey, ez, bx, by, bz, tau, tc, s_qs, s_bw, tab, dt,
                              sg.proc == QED_PROC_QS ? cut_qs : cut_bw, stats, dry, bad);
    }
    if (!dry) warp_count_err(stats ? stats + QED_STAT_NONFINITE : nullptr, bad, QED_EW_NONFINITE);
}

// 15 consumer warps + the producer (16 warps, one CTA per SM), 2 stages, as the single-call default
constexpr int kSegBulkCW = 15, kSegBulkS = 2;

static qed_status launch_evolve_seg_bulk(const EvolveSeg<float> *segs, int n_seg, const TablesView<float> &tab,
                                         float dt, float cut_qs, float cut_bw, long long *stats, int dry,
                                         long long wait_cycles, cudaStream_t st)
{
    constexpr size_t stage = (size_t)kSegBulkS * kSegArrays * kSegBulkCW * 32 * 4 * sizeof(float);
    const size_t dyn = stage + (size_t)n_seg * 2 * sizeof(long long);
    auto k = evolve_seg_bulk_kernel<kSegBulkCW, kSegBulkS>;
    static bool attr = false;
    if (!attr) {
        QED_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)(stage + 3 * QED_MAX_PATCHES * 2 * sizeof(long long))));
        attr = true;
    }
    k<<<sm_count(), (kSegBulkCW + 1) * 32, dyn, st>>>(segs, n_seg, tab, dt, cut_qs, cut_bw, stats, dry,
                                                       wait_cycles);
    QED_LAUNCH_CHECK();
    return QED_OK;
}

// CTAs of 256 threads for `warps` warp chunks of work, at most the resident count
static int resident_grid(int64_t warps, int per_sm)
{
    int64_t grid = (warps + 7) / 8;
    const int64_t cap = (int64_t)sm_count() * (per_sm > 0 ? per_sm : 1);
    return (int)(grid < 1 ? 1 : (grid > cap ? cap : grid));
}

template <typename T, bool QS>
static qed_status launch_events_batched(const qed_batch *b, const EventCommon<T> &c, bool mlp, cudaStream_t st)
{
    const int n_seg = QS ? 2 * b->n_patches : b->n_patches;
    const EventSeg<T> *segs = (const EventSeg<T> *)(QS ? b->d_qs : b->d_bw);
    const size_t dyn = (mlp ? sizeof(InferSmem) : 0) + (size_t)n_seg * 2 * sizeof(long long);
    const int64_t warps = (b->fire_capacity_max * (QS ? 2 : 1) + 31) / 32;
    // the opt-in shared-memory size is set once, for the largest batch; the grid
    // is at most what stays resident (every CTA strides over the chunks)
    constexpr int kMaxDyn = (int)sizeof(InferSmem) + 2 * QED_MAX_PATCHES * 2 * (int)sizeof(long long);
    if (mlp) {
        auto k = event_batched_kernel<T, true, QS>;
        static bool attr = false;
        static int per_sm = 0;
        if (!attr) {
            QED_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDyn));
            QED_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, kMaxDyn));
            attr = true;
        }
        k<<<resident_grid(warps, per_sm), 256, dyn, st>>>(segs, n_seg, c);
    } else {
        auto k = event_batched_kernel<T, false, QS>;
        static bool attr = false;
        static int per_sm = 0;
        if (!attr) {
            QED_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDyn));
            QED_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, 2 * QED_MAX_PATCHES * 2 *
                                                                                      (int)sizeof(long long)));
            attr = true;
        }
        k<<<resident_grid(warps, per_sm), 256, dyn, st>>>(segs, n_seg, c);
    }
    QED_LAUNCH_CHECK();
    return QED_OK;
}

template <typename T>
static qed_status launch_events_batched_all(const qed_batch *b, const EventCommon<T> &cq, const EventCommon<T> &cb,
                                           cudaStream_t st)
{
    const int n_qs = 2 * b->n_patches, n_bw = b->n_patches;
    const size_t dyn = (size_t)(n_qs + n_bw) * 2 * sizeof(long long);
    const int64_t warps = (b->fire_capacity_max * 3 + 31) / 32;
    constexpr int kMaxDyn = 3 * QED_MAX_PATCHES * 2 * (int)sizeof(long long);
    auto k = event_batched_all_kernel<T>;
    static bool attr = false;
    static int per_sm = 0;
    if (!attr) {
        QED_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDyn));
        QED_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, kMaxDyn));
        attr = true;
    }
    k<<<resident_grid(warps, per_sm), 256, dyn, st>>>((const EventSeg<T> *)b->d_qs, n_qs,
                                                      (const EventSeg<T> *)b->d_bw, n_bw, cq, cb);
    QED_LAUNCH_CHECK();
    return QED_OK;
}

template <typename T>
static qed_status build_batch(const qed_patch *patches, int n, qed_batch *b, cudaStream_t st)
{
    std::vector<EvolveSeg<T>> ev(3 * (size_t)n);
    std::vector<EventSeg<T>> qs(2 * (size_t)n), bw((size_t)n);
    std::vector<int64_t *> zero(3 * (size_t)n);
    std::vector<ClampEntry> clamp(6 * (size_t)n);
    bool vec = true;
    int64_t capsum = 0, fmax = 0;
    for (int i = 0; i < n; ++i) {
        const qed_patch &p = patches[i];
        const qed_species *sp[3] = {&p.electrons, &p.positrons, &p.photons};
        const int proc[3] = {QED_PROC_QS, QED_PROC_QS, QED_PROC_BW};
        for (int k = 0; k < 3; ++k) {
            vec = fill_seg<T>(ev[3 * i + k], sp[k], proc[k], &p.fire[k]) && vec;
            zero[3 * i + k] = p.fire[k].d_count;
            clamp[6 * i + k] = ClampEntry{(unsigned long long *)sp[k]->d_count, sp[k]->capacity};
            clamp[6 * i + 3 + k] = ClampEntry{(unsigned long long *)p.fire[k].d_count, p.fire[k].capacity};
            capsum += sp[k]->capacity;
            fmax = fmax > p.fire[k].capacity ? fmax : p.fire[k].capacity;
        }
        for (int k = 0; k < 2; ++k) {
            EventSeg<T> &g = qs[2 * i + k];
            memset(&g, 0, sizeof(g));
            g.parent = ptrs<T>(sp[k]);
            g.out0 = ptrs<T>(&p.photons);
            g.fire_idx = p.fire[k].idx, g.fire_chi = p.fire[k].chi, g.fire_count = p.fire[k].d_count;
            g.fire_cap = p.fire[k].capacity;
        }
        EventSeg<T> &g = bw[i];
        memset(&g, 0, sizeof(g));
        g.parent = ptrs<T>(&p.photons);
        g.out0 = ptrs<T>(&p.electrons);
        g.out1 = ptrs<T>(&p.positrons);
        g.fire_idx = p.fire[2].idx, g.fire_chi = p.fire[2].chi, g.fire_count = p.fire[2].d_count;
        g.fire_cap = p.fire[2].capacity;
    }
    bool positions = true, pos_al16 = true;
    std::vector<PushSeg<T>> push(3 * (size_t)n);
    for (int i = 0; i < n; ++i) {
        const qed_species *sp[3] = {&patches[i].electrons, &patches[i].positrons, &patches[i].photons};
        const double q[3] = {-1.0, 1.0, 0.0};
        for (int k = 0; k < 3; ++k) {
            positions = positions && sp[k]->x && sp[k]->y && sp[k]->z;
            for (const void *a : {sp[k]->x, sp[k]->y, sp[k]->z})
                pos_al16 = pos_al16 && ((uintptr_t)a & 15u) == 0;
            push[3 * i + k] = push_seg<T>(sp[k], q[k]);
        }
    }
    if (positions) {
        QED_CUDA_TRY(cudaMalloc(&b->d_push, push.size() * sizeof(PushSeg<T>)));
        QED_CUDA_TRY(cudaMemcpyAsync(b->d_push, push.data(), push.size() * sizeof(PushSeg<T>), cudaMemcpyHostToDevice,
                                     st));
    }
    struct Up {
        void **dst;
        const void *src;
        size_t bytes;
    } ups[5] = {{&b->d_evolve, ev.data(), ev.size() * sizeof(EvolveSeg<T>)},
                {&b->d_qs, qs.data(), qs.size() * sizeof(EventSeg<T>)},
                {&b->d_bw, bw.data(), bw.size() * sizeof(EventSeg<T>)},
                {(void **)&b->d_zero, zero.data(), zero.size() * sizeof(int64_t *)},
                {(void **)&b->d_clamp, clamp.data(), clamp.size() * sizeof(ClampEntry)}};
    for (const Up &u : ups) {
        QED_CUDA_TRY(cudaMalloc(u.dst, u.bytes));
        QED_CUDA_TRY(cudaMemcpyAsync(*u.dst, u.src, u.bytes, cudaMemcpyHostToDevice, st));
    }
    QED_CUDA_TRY(cudaStreamSynchronize(st));
    b->vec = vec;
    b->push_vec = vec && positions && pos_al16;
    b->capacity_sum = capsum;
    b->fire_capacity_max = fmax;
    return QED_OK;
}

// wave != NULL: the push in that wave is fused into the evolution (one pass
// per particle), at time t0 + step * dt (step from opts->d_step when set)
template <typename T>
static qed_status substep_batched_impl(const qed_tables *t, const qed_batch *b, double dt, uint64_t seed, int64_t step,
                                       const qed_substep_opts *o, cudaStream_t st, const qed_plane_wave *wave = nullptr,
                                       double t0 = 0.0, int store_fields = 0)
{
    const int n = b->n_patches;
    long long *stats = o ? (long long *)o->d_stats : nullptr;
    zero_counts_kernel<<<1, 256, 0, st>>>(b->d_zero, 3 * n, b->d_clamp, n, stats);
    QED_LAUNCH_CHECK();
    const int threads = (o && o->evolve_threads) ? o->evolve_threads : (b->threads ? b->threads : 256);
    const int ctas = (o && o->evolve_ctas_per_sm) ? o->evolve_ctas_per_sm : b->ctas_per_sm;
    // the default shape (nothing asked for, nothing tuned) of an FP32 batch with
    // aligned arrays: the bulk-copy kernel
    const bool bulk = sizeof(T) == 4 && b->vec && !(o && (o->evolve_threads || o->evolve_ctas_per_sm)) &&
                      !(o && o->evolve_pipeline == QED_EVOLVE_DIRECT) && b->threads == 0 && b->ctas_per_sm == 0;
    if (o && o->evolve_begin) QED_CUDA_TRY(cudaEventRecord((cudaEvent_t)o->evolve_begin, st));
    const T cut_qs = o ? (T)o->qs_chi_cut : T(0), cut_bw = o ? (T)o->bw_chi_cut : T(0);
    qed_status s;
    if (wave) {
        s = launch_push_evolve<T>((const EvolveSeg<T> *)b->d_evolve, b->d_push, 3 * n, make_view<T>(t),
                                  wave_params(wave), t0, dt, o ? o->d_step : nullptr, step, cut_qs, cut_bw, stats,
                                  store_fields, b->push_vec, st);
    } else if constexpr (sizeof(T) == 4) {
        s = bulk ? launch_evolve_seg_bulk((const EvolveSeg<float> *)b->d_evolve, 3 * n, make_view<float>(t),
                                          (float)dt, cut_qs, cut_bw, stats, 0, o ? o->wait_limit_cycles : 0, st)
                 : launch_evolve_segments<T>((const EvolveSeg<T> *)b->d_evolve, 3 * n, make_view<T>(t), (T)dt,
                                             cut_qs, cut_bw, stats, 0, b->vec, threads, ctas, st);
    } else {
        s = launch_evolve_segments<T>((const EvolveSeg<T> *)b->d_evolve, 3 * n, make_view<T>(t), (T)dt, cut_qs,
                                      cut_bw, stats, 0, b->vec, threads, ctas, st);
    }
    if (s) return s;
    if (o && o->evolve_end) QED_CUDA_TRY(cudaEventRecord((cudaEvent_t)o->evolve_end, st));
    const bool mlp = o && o->sampler == 1;
    if (mlp) {
        if ((s = launch_events_batched<T, false>(b, event_common<T>(t, QED_PROC_BW, seed, step, o), true, st)))
            return s;
        if ((s = launch_events_batched<T, true>(b, event_common<T>(t, QED_PROC_QS, seed, step, o), true, st)))
            return s;
    } else {
        // the push fused into the evolution without stored fields computes every
        // particle's fields itself: the photons emitted get none
        EventCommon<T> cq = event_common<T>(t, QED_PROC_QS, seed, step, o);
        cq.copy_fields = (wave && !store_fields) ? 0 : 1;
        if ((s = launch_events_batched_all<T>(b, cq, event_common<T>(t, QED_PROC_BW, seed, step, o), st))) return s;
    }
    clamp_batch_kernel<<<(6 * n + 255) / 256, 256, 0, st>>>(b->d_clamp, 6 * n, o ? o->d_step : nullptr);
    QED_LAUNCH_CHECK();
    return QED_OK;
}

static void free_batch(qed_batch *b)
{
    if (!b) return;
    void *p[] = {b->d_evolve, b->d_qs, b->d_bw, b->d_zero, b->d_clamp, b->d_push};
    for (void *x : p)
        if (x) cudaFree(x);
    delete b;
}

}  // namespace qed

using namespace qed;

extern "C" qed_status qed_batch_create(const qed_patch *patches, int32_t n_patches, qed_precision prec,
                                       qed_batch **out, void *stream)
{
    clear_error();
    if (!out) QED_FAIL(QED_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!patches || n_patches <= 0 || n_patches > QED_MAX_PATCHES)
        QED_FAIL(QED_ERR_INVALID_ARG, "need 1 <= n_patches <= %d (got %d)", QED_MAX_PATCHES, (int)n_patches);
    qed_status s;
    for (int i = 0; i < n_patches; ++i) {
        if ((s = check_species(&patches[i].electrons, "electrons", prec))) return s;
        if ((s = check_species(&patches[i].positrons, "positrons", prec))) return s;
        if ((s = check_species(&patches[i].photons, "photons", prec))) return s;
        for (int k = 0; k < 3; ++k)
            if ((s = check_fire(&patches[i].fire[k], "fire"))) return s;
    }
    qed_batch *b = new qed_batch();
    memset(b, 0, sizeof(*b));
    cudaGetDevice(&b->device);
    b->prec = prec;
    b->n_patches = n_patches;
    cudaStream_t st = as_stream(stream);
    s = prec == QED_F32 ? build_batch<float>(patches, n_patches, b, st)
                        : build_batch<double>(patches, n_patches, b, st);
    if (s) {
        free_batch(b);
        return s;
    }
    *out = b;
    return QED_OK;
}

extern "C" qed_status qed_batch_destroy(qed_batch *b)
{
    clear_error();
    free_batch(b);
    return QED_OK;
}

extern "C" qed_status qed_substep_batched(const qed_tables *t, const qed_batch *b, double dt, uint64_t seed,
                                          int64_t step, const qed_substep_opts *opts, void *stream)
{
    clear_error();
    qed_status s;
    if ((s = check_tables(t))) return s;
    if (!b) QED_FAIL(QED_ERR_INVALID_ARG, "batch is NULL");
    if ((s = check_opts(opts))) return s;
    if (!std::isfinite(dt) || dt < 0) QED_FAIL(QED_ERR_INVALID_ARG, "dt must be finite and >= 0");
    if (opts && opts->evolve_threads && opts->evolve_threads != 128 && opts->evolve_threads != 256 &&
        opts->evolve_threads != 512)
        QED_FAIL(QED_ERR_INVALID_ARG, "evolve_threads must be 128, 256 or 512");
    if (opts && (opts->evolve_ctas_per_sm < 0 || opts->evolve_ctas_per_sm > 8))
        QED_FAIL(QED_ERR_INVALID_ARG, "evolve_ctas_per_sm must be in [0, 8]");
    cudaStream_t st = as_stream(stream);
    return b->prec == QED_F32 ? substep_batched_impl<float>(t, b, dt, seed, step, opts, st)
                              : substep_batched_impl<double>(t, b, dt, seed, step, opts, st);
}

extern "C" qed_status qed_push_substep_batched(const qed_tables *t, const qed_batch *b, const qed_plane_wave *wave,
                                               double t0, double dt, uint64_t seed, int64_t step,
                                               const qed_substep_opts *opts, int32_t store_fields, void *stream)
{
    clear_error();
    qed_status s;
    if ((s = check_tables(t))) return s;
    if (!b) QED_FAIL(QED_ERR_INVALID_ARG, "batch is NULL");
    if (!b->d_push) QED_FAIL(QED_ERR_INVALID_ARG, "the batch's species have no positions");
    if ((s = check_wave(wave))) return s;
    if ((s = check_opts(opts))) return s;
    if (!std::isfinite(dt) || dt < 0) QED_FAIL(QED_ERR_INVALID_ARG, "dt must be finite and >= 0");
    if (!std::isfinite(t0)) QED_FAIL(QED_ERR_INVALID_ARG, "t0 must be finite");
    cudaStream_t st = as_stream(stream);
    return b->prec == QED_F32
               ? substep_batched_impl<float>(t, b, dt, seed, step, opts, st, wave, t0, store_fields != 0)
               : substep_batched_impl<double>(t, b, dt, seed, step, opts, st, wave, t0, store_fields != 0);
}

extern "C" qed_status qed_tune_evolve(const qed_tables *t, qed_batch *b, int32_t *threads_out,
                                      int32_t *ctas_per_sm_out, float *ms_out, void *stream)
{
    clear_error();
    qed_status s;
    if ((s = check_tables(t))) return s;
    if (!b) QED_FAIL(QED_ERR_INVALID_ARG, "batch is NULL");
    cudaStream_t st = as_stream(stream);
    cudaEvent_t e0, e1;
    QED_CUDA_TRY(cudaEventCreate(&e0));
    QED_CUDA_TRY(cudaEventCreate(&e1));
    const int cand_threads[3] = {128, 256, 512};
    float best = 1e30f;
    int bt = 256, bc = 0;
    if (b->prec == QED_F32 && b->vec) {  // the default: the bulk-copy kernel (reported as 0, 0)
        float tot = 0.f;
        for (int rep = 0; rep < 4 && s == QED_OK; ++rep) {
            cudaEventRecord(e0, st);
            s = launch_evolve_seg_bulk((const EvolveSeg<float> *)b->d_evolve, 3 * b->n_patches, make_view<float>(t),
                                       0.f, 0.f, 0.f, nullptr, 1, 0, st);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) tot += ms;
        }
        if (s == QED_OK) best = tot / 3, bt = 0, bc = 0;
    }
    for (int th : cand_threads) {
        const int max_ctas = 768 / th;  // the register budget of the kernel's launch bounds
        for (int c = 1; c <= max_ctas && s == QED_OK; ++c) {
            float tot = 0.f;
            for (int rep = 0; rep < 4 && s == QED_OK; ++rep) {
                cudaEventRecord(e0, st);
                s = b->prec == QED_F32
                        ? launch_evolve_segments<float>((const EvolveSeg<float> *)b->d_evolve, 3 * b->n_patches,
                                                        make_view<float>(t), 0.f, 0.f, 0.f, nullptr, 1, b->vec, th,
                                                        c, st)
                        : launch_evolve_segments<double>((const EvolveSeg<double> *)b->d_evolve, 3 * b->n_patches,
                                                         make_view<double>(t), 0.0, 0.0, 0.0, nullptr, 1, b->vec, th,
                                                         c, st);
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) tot += ms;  // the first run warms up
            }
            if (s == QED_OK && tot / 3 < best) best = tot / 3, bt = th, bc = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s) return s;
    b->threads = bt;
    b->ctas_per_sm = bc;
    if (threads_out) *threads_out = bt;
    if (ctas_per_sm_out) *ctas_per_sm_out = bc;
    if (ms_out) *ms_out = best;
    return QED_OK;
}

extern "C" qed_status qed_push_batched(const qed_batch *b, const qed_plane_wave *wave, double t0, double dt,
                                       int64_t step, const int64_t *d_step, void *stream)
{
    clear_error();
    qed_status s;
    if (!b) QED_FAIL(QED_ERR_INVALID_ARG, "batch is NULL");
    if (!b->d_push) QED_FAIL(QED_ERR_INVALID_ARG, "the batch's species have no positions");
    if ((s = check_wave(wave))) return s;
    if (!std::isfinite(dt) || dt < 0) QED_FAIL(QED_ERR_INVALID_ARG, "dt must be finite and >= 0");
    cudaStream_t st = as_stream(stream);
    return b->prec == QED_F32
               ? launch_push<float>(b->d_push, 3 * b->n_patches, wave_params(wave), t0, dt, d_step, step,
                                    b->capacity_sum, st)
               : launch_push<double>(b->d_push, 3 * b->n_patches, wave_params(wave), t0, dt, d_step, step,
                                     b->capacity_sum, st);
}
