// evolve.cu -- optical-depth evolution (§3, Fig. scheme) as one batched,
// persistent launch over many particle segments (species or patches), with
// warp-ballot compaction of the firing particles, plus the optical-depth
// initialisation.
//
// Layout: every segment is a structure of arrays in HBM.  A CTA walks tiles of
// (256 threads x VEC) consecutive particles of one segment; each thread loads
// VEC particles with one 16-byte load per component (float4 / double2), keeps
// the 1-D rate tables of both processes in shared memory, and writes back only
// the optical depth (and its Kahan word in FP32).  Tiles of all segments form
// one index space; CTAs stride over it, so uneven segment sizes share the grid.
#include <algorithm>

#include "launch.cuh"
#include "evolve_core.cuh"
#include "pipeline.cuh"

namespace qed {

// One tile: THREADS x VEC consecutive particles of segment `sg` starting at
// tile index `first`, loaded straight from global memory.
template <typename T, int VEC, int THREADS>
__device__ __forceinline__ void evolve_tile(const EvolveSeg<T> &sg, int64_t n, long long first, const T *s_qs,
                                            const T *s_bw, const TablesView<T> &tab, T dt, T cut, long long *stats,
                                            int dry, int &bad)
{
    const int64_t i0 = first * ((int64_t)THREADS * VEC) + (int64_t)threadIdx.x * VEC;
    T px[VEC], py[VEC], pz[VEC], ex[VEC], ey[VEC], ez[VEC], bx[VEC], by[VEC], bz[VEC], tau[VEC], tc[VEC];
    const bool full = i0 + VEC <= n;
    if (full) {
        load_vec<T, VEC>(sg.px, i0, px);
        load_vec<T, VEC>(sg.py, i0, py);
        load_vec<T, VEC>(sg.pz, i0, pz);
        load_vec<T, VEC>(sg.ex, i0, ex);
        load_vec<T, VEC>(sg.ey, i0, ey);
        load_vec<T, VEC>(sg.ez, i0, ez);
        load_vec<T, VEC>(sg.bx, i0, bx);
        load_vec<T, VEC>(sg.by, i0, by);
        load_vec<T, VEC>(sg.bz, i0, bz);
        load_vec<T, VEC>(sg.tau, i0, tau);
        if constexpr (sizeof(T) == 4) load_vec<T, VEC>(sg.tau_c, i0, tc);
    } else {
        load_scalar<T, VEC>(sg, n, i0, px, py, pz, ex, ey, ez, bx, by, bz, tau, tc);
    }
    evolve_regs<T, VEC>(sg, n, i0, full, px, py, pz, ex, ey, ez, bx, by, bz, tau, tc, s_qs, s_bw, tab, dt, cut,
                        stats, dry, bad);
}

// the k-th streamed array of a segment: px .. bz, tau, tau_c
template <typename T>
__device__ __forceinline__ const T *seg_array(const EvolveSeg<T> &g, int k)
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

// segments as kernel parameters (a few species); MINB resident CTAs per SM
template <typename T, int VEC, int MAXSEG, int MINB = 3>
__global__ void __launch_bounds__(kEvolveThreads, MINB)
    evolve_kernel(const __grid_constant__ EvolveArgs<T, MAXSEG> a)
{
    __shared__ T s_qs[QED_MAX_TABLE_N];
    __shared__ T s_bw[QED_MAX_TABLE_N];
    __shared__ long long s_end[MAXSEG];  // inclusive prefix of tile counts
    __shared__ long long s_n[MAXSEG];
    constexpr int64_t tile = kEvolveTile<T, VEC>;

    for (int i = threadIdx.x; i < a.tab.qs_G.n; i += blockDim.x) s_qs[i] = a.tab.qs_G.ln_f[i];
    for (int i = threadIdx.x; i < a.tab.bw_T.n; i += blockDim.x) s_bw[i] = a.tab.bw_T.ln_f[i];
    if (threadIdx.x == 0) {
        long long acc = 0;
        for (int s = 0; s < a.n_seg; ++s) {
            long long n = *a.seg[s].count;
            n = n < 0 ? 0 : (n > a.seg[s].capacity ? a.seg[s].capacity : n);
            s_n[s] = n;
            acc += (n + tile - 1) / tile;
            s_end[s] = acc;
        }
    }
    __syncthreads();
    const long long total = a.n_seg ? s_end[a.n_seg - 1] : 0;
    int bad = 0;
    for (long long t = blockIdx.x; t < total; t += gridDim.x) {
        int s = 0;
        while (t >= s_end[s]) ++s;
        evolve_tile<T, VEC, kEvolveThreads>(a.seg[s], s_n[s], t - (s ? s_end[s - 1] : 0), s_qs, s_bw, a.tab, a.dt,
                                            a.chi_cut[a.seg[s].proc], a.stats, 0, bad);
    }
    warp_count_err(a.stats ? a.stats + QED_STAT_NONFINITE : nullptr, bad, QED_EW_NONFINITE);
}

// ---------------------------------------------------------------------------
// Bulk-copy pipeline (FP32, 16-byte-aligned arrays).  The last warp of the CTA
// is the producer: for every full tile of TP = CW x 32 x 4 particles, eleven of
// its lanes each issue one cp.async.bulk of that tile of one array (px .. bz,
// tau, tau_c; TP x 4 bytes) into a shared-memory stage, counted on the stage's
// `full` mbarrier.  The CW consumer warps read the stage with conflict-free
// float4 loads (4 consecutive particles per thread), release it on the `empty`
// mbarrier (one arrival per warp) before they compute, evaluate, and store the
// optical depths with 16-byte streaming stores.  The ragged last tile of a
// segment is not copied: its consumers load it from global memory.  S stages
// keep S - 1 tiles of every SM's stream in flight while one is evaluated.
// ---------------------------------------------------------------------------
constexpr int kBulkArrays = 11;

// bounded wait (limit cycles) that also gives up as soon as another warp has given up
__device__ __forceinline__ bool bulk_wait(uint64_t *bar, uint32_t parity, volatile int *abort, long long limit)
{
    if (limit < kWaitCycles) {
        // a caller's shorter limit: probe without the hardware's suspended wait,
        // which by itself can outlast a limit of a few cycles
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

__device__ __forceinline__ void bulk_give_up(int *abort, long long *stats)
{
    if (atomicExch(abort, 1) == 0) {
        note_error(QED_EW_WAIT_TIMEOUT);
        if (stats) atomicAdd((unsigned long long *)(stats + QED_STAT_WAIT_TIMEOUT), 1ull);
    }
}

template <int CW, int S>
constexpr size_t kBulkStageBytes = (size_t)S * kBulkArrays * CW * 32 * 4 * sizeof(float);

template <int CW, int S, int MINB, int MAXSEG>
__global__ void __launch_bounds__((CW + 1) * 32, MINB)
    evolve_bulk_kernel(const __grid_constant__ EvolveArgs<float, MAXSEG> a)
{
    constexpr int TP = CW * 32 * 4;
    extern __shared__ __align__(128) float s_stage[];  // [S][kBulkArrays][TP]
    __shared__ __align__(8) uint64_t s_full[S];
    __shared__ __align__(8) uint64_t s_empty[S];
    __shared__ float s_qs[QED_MAX_TABLE_N];
    __shared__ float s_bw[QED_MAX_TABLE_N];
    __shared__ long long s_end[MAXSEG];
    __shared__ long long s_n[MAXSEG];
    __shared__ int s_abort;

    for (int i = threadIdx.x; i < a.tab.qs_G.n; i += blockDim.x) s_qs[i] = a.tab.qs_G.ln_f[i];
    for (int i = threadIdx.x; i < a.tab.bw_T.n; i += blockDim.x) s_bw[i] = a.tab.bw_T.ln_f[i];
    if (threadIdx.x == 0) {
        long long acc = 0;
        for (int s = 0; s < a.n_seg; ++s) {
            long long n = *a.seg[s].count;
            n = n < 0 ? 0 : (n > a.seg[s].capacity ? a.seg[s].capacity : n);
            s_n[s] = n;
            acc += (n + TP - 1) / TP;
            s_end[s] = acc;
        }
        s_abort = 0;
        for (int k = 0; k < S; ++k) {
            mbar_init(&s_full[k], 1);
            mbar_init(&s_empty[k], CW);
        }
        mbar_fence_init();
    }
    __syncthreads();
    const long long total = a.n_seg ? s_end[a.n_seg - 1] : 0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int *abort = &s_abort;
    // the producer/consumer hand-offs use the caller's limit; the final wait for
    // the copies in flight (below) always the full one
    const long long limit = a.wait_cycles > 0 ? a.wait_cycles : kWaitCycles;

    if (warp == CW) {  // producer
        const uint64_t pol = l2_evict_first();
        int k = 0;
        for (long long t = blockIdx.x; t < total; t += gridDim.x, ++k) {
            const int st = k % S;
            const uint32_t ph = (uint32_t)(k / S) & 1u;
            int s = 0;
            while (t >= s_end[s]) ++s;
            const int64_t i0 = (t - (s ? s_end[s - 1] : 0)) * (int64_t)TP;
            const bool ok = __all_sync(0xffffffffu, bulk_wait(&s_empty[st], ph ^ 1u, abort, limit));
            if (!ok) {
                if (lane == 0) bulk_give_up(&s_abort, a.stats);
                break;
            }
            if (i0 + TP <= s_n[s]) {
                if (lane == 0) mbar_arrive_expect_tx(&s_full[st], kBulkArrays * TP * (uint32_t)sizeof(float));
                __syncwarp();
                if (lane < kBulkArrays)
                    bulk_g2s(s_stage + ((size_t)st * kBulkArrays + lane) * TP, seg_array<float>(a.seg[s], lane) + i0,
                             TP * (uint32_t)sizeof(float), &s_full[st], pol);
            } else if (lane == 0) {
                mbar_arrive(&s_full[st]);
            }
        }
        // leave only once the copies of the last S tiles have landed
        for (int j = 1; j <= S && j <= k; ++j) {
            const int kk = k - j;
            if (!mbar_wait(&s_full[kk % S], (uint32_t)(kk / S) & 1u) && lane == 0) bulk_give_up(&s_abort, a.stats);
        }
        return;
    }

    int bad = 0;
    int k = 0;
    for (long long t = blockIdx.x; t < total; t += gridDim.x, ++k) {
        const int st = k % S;
        const uint32_t ph = (uint32_t)(k / S) & 1u;
        int s = 0;
        while (t >= s_end[s]) ++s;
        const EvolveSeg<float> &sg = a.seg[s];
        const int64_t n = s_n[s];
        const int64_t base = (t - (s ? s_end[s - 1] : 0)) * (int64_t)TP;
        const int64_t i0 = base + 4 * (int64_t)threadIdx.x;
        const bool ok = __all_sync(0xffffffffu, bulk_wait(&s_full[st], ph, abort, limit));
        if (!ok) {
            if (lane == 0) bulk_give_up(&s_abort, a.stats);
            break;
        }
        float px[4], py[4], pz[4], ex[4], ey[4], ez[4], bx[4], by[4], bz[4], tau[4], tc[4];
        bool full4;
        if (base + TP <= n) {
            const float4 *v = reinterpret_cast<const float4 *>(s_stage + (size_t)st * kBulkArrays * TP) + threadIdx.x;
            constexpr int q = TP / 4;
            float4 w;
#define QED_UNPACK(arr, k)                                 \
    w = v[(k) * q];                                        \
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
        evolve_regs<float, 4>(sg, n, i0, full4, px, py, pz, ex, ey, ez, bx, by, bz, tau, tc, s_qs, s_bw, a.tab,
                              a.dt, a.chi_cut[sg.proc], a.stats, 0, bad);
    }
    warp_count_err(a.stats ? a.stats + QED_STAT_NONFINITE : nullptr, bad, QED_EW_NONFINITE);
}

template <int CW, int S, int MINB, int MAXSEG>
static qed_status launch_bulk(const EvolveArgs<float, MAXSEG> &a, int64_t capacity_sum, cudaStream_t st)
{
    constexpr size_t dyn = kBulkStageBytes<CW, S>;
    static bool attr = false;
    if (!attr) {
        QED_CUDA_TRY(cudaFuncSetAttribute(evolve_bulk_kernel<CW, S, MINB, MAXSEG>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
        attr = true;
    }
    constexpr int64_t tp = (int64_t)CW * 32 * 4;
    const int64_t tiles = (capacity_sum + tp - 1) / tp;
    int64_t g = (int64_t)sm_count() * MINB;
    if (tiles < g) g = tiles < 1 ? 1 : tiles;
    evolve_bulk_kernel<CW, S, MINB, MAXSEG><<<(int)g, (CW + 1) * 32, dyn, st>>>(a);
    QED_LAUNCH_CHECK();
    return QED_OK;
}

// Segments in device memory (many patches): every CTA reads all segment
// counts, forms the prefix sum of their tile counts in shared memory (a block
// scan), and strides over the combined tile space; a tile's segment is found
// by binary search.
template <typename T, int VEC, int THREADS>
__global__ void __launch_bounds__(THREADS, 768 / THREADS)
    evolve_seg_kernel(const EvolveSeg<T> *__restrict__ segs, int n_seg, TablesView<T> tab, T dt, T cut_qs, T cut_bw,
                      long long *stats, int dry)
{
    __shared__ T s_qs[QED_MAX_TABLE_N];
    __shared__ T s_bw[QED_MAX_TABLE_N];
    __shared__ long long s_warp[THREADS / 32];
    extern __shared__ long long s_dyn[];  // [n_seg] inclusive tile prefix, [n_seg] counts
    long long *s_end = s_dyn, *s_n = s_dyn + n_seg;
    constexpr int64_t tile = (int64_t)THREADS * VEC;

    for (int i = threadIdx.x; i < tab.qs_G.n; i += THREADS) s_qs[i] = tab.qs_G.ln_f[i];
    for (int i = threadIdx.x; i < tab.bw_T.n; i += THREADS) s_bw[i] = tab.bw_T.ln_f[i];
    const long long total = tile_prefix<T, THREADS>(segs, n_seg, tile, s_end, s_n, s_warp);
    int bad = 0;
    for (long long t = blockIdx.x; t < total; t += gridDim.x) {
        const int lo = find_segment(s_end, n_seg, t);
        const EvolveSeg<T> &sg = segs[lo];
        evolve_tile<T, VEC, THREADS>(sg, s_n[lo], t - (lo ? s_end[lo - 1] : 0), s_qs, s_bw, tab, dt,
                                     sg.proc == QED_PROC_QS ? cut_qs : cut_bw, stats, dry, bad);
    }
    if (!dry) warp_count_err(stats ? stats + QED_STAT_NONFINITE : nullptr, bad, QED_EW_NONFINITE);
}

template <typename T, int THREADS>
static qed_status launch_seg_impl(const EvolveSeg<T> *segs, int n_seg, const TablesView<T> &tab, T dt, T cut_qs,
                                  T cut_bw, long long *stats, int dry, bool vec, int ctas_per_sm, cudaStream_t st)
{
    const size_t dyn = (size_t)n_seg * 2 * sizeof(long long);
    int grid = sm_count() * (ctas_per_sm > 0 ? ctas_per_sm : 768 / THREADS);
    // the opt-in shared-memory size is set once per kernel, for the largest batch
    constexpr int kMaxDyn = 3 * QED_MAX_PATCHES * 2 * (int)sizeof(long long);
    if (vec) {
        constexpr int V = sizeof(T) == 4 ? 4 : 2;
        static bool attr = false;
        if (!attr) {
            QED_CUDA_TRY(cudaFuncSetAttribute(evolve_seg_kernel<T, V, THREADS>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDyn));
            attr = true;
        }
        evolve_seg_kernel<T, V, THREADS><<<grid, THREADS, dyn, st>>>(segs, n_seg, tab, dt, cut_qs, cut_bw, stats,
                                                                      dry);
    } else {
        static bool attr = false;
        if (!attr) {
            QED_CUDA_TRY(cudaFuncSetAttribute(evolve_seg_kernel<T, 1, THREADS>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDyn));
            attr = true;
        }
        evolve_seg_kernel<T, 1, THREADS><<<grid, THREADS, dyn, st>>>(segs, n_seg, tab, dt, cut_qs, cut_bw, stats,
                                                                      dry);
    }
    QED_LAUNCH_CHECK();
    return QED_OK;
}

template <typename T>
qed_status launch_evolve_segments(const EvolveSeg<T> *d_segs, int n_seg, const TablesView<T> &tab, T dt, T cut_qs,
                                  T cut_bw, long long *stats, int dry, bool vec, int threads, int ctas_per_sm,
                                  cudaStream_t st)
{
    if (n_seg <= 0) return QED_OK;
    switch (threads) {
    case 128:
        return launch_seg_impl<T, 128>(d_segs, n_seg, tab, dt, cut_qs, cut_bw, stats, dry, vec, ctas_per_sm, st);
    case 512:
        return launch_seg_impl<T, 512>(d_segs, n_seg, tab, dt, cut_qs, cut_bw, stats, dry, vec, ctas_per_sm, st);
    default:
        return launch_seg_impl<T, 256>(d_segs, n_seg, tab, dt, cut_qs, cut_bw, stats, dry, vec, ctas_per_sm, st);
    }
}

template qed_status launch_evolve_segments<float>(const EvolveSeg<float> *, int, const TablesView<float> &, float,
                                                  float, float, long long *, int, bool, int, int, cudaStream_t);
template qed_status launch_evolve_segments<double>(const EvolveSeg<double> *, int, const TablesView<double> &,
                                                   double, double, double, long long *, int, bool, int, int,
                                                   cudaStream_t);

// clamp the firing counters to their capacity once the evolution is done
__global__ void clamp_fire_counts(unsigned long long *c0, int64_t cap0, unsigned long long *c1, int64_t cap1,
                                  unsigned long long *c2, int64_t cap2)
{
    if (threadIdx.x == 0) {
        if (c0 && *c0 > (unsigned long long)cap0) *c0 = cap0;
        if (c1 && *c1 > (unsigned long long)cap1) *c1 = cap1;
        if (c2 && *c2 > (unsigned long long)cap2) *c2 = cap2;
    }
}

static int g_sm_count = 0;

int sm_count()
{
    if (g_sm_count == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev);
        if (g_sm_count <= 0) g_sm_count = 1;
    }
    return g_sm_count;
}

template <typename T, int VEC, int MAXSEG, int MINB = 3>
static int evolve_grid(int64_t total_particles)
{
    static int blocks_per_sm = 0;
    if (blocks_per_sm == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, evolve_kernel<T, VEC, MAXSEG, MINB>,
                                                      kEvolveThreads, 0);
        if (blocks_per_sm <= 0) blocks_per_sm = 1;
    }
    const int64_t tiles = (total_particles + kEvolveTile<T, VEC> - 1) / kEvolveTile<T, VEC>;
    int64_t g = (int64_t)sm_count() * blocks_per_sm;
    if (tiles < g) g = tiles < 1 ? 1 : tiles;
    return (int)g;
}

template <typename T, int MAXSEG>
qed_status launch_evolve(const EvolveArgs<T, MAXSEG> &a, bool vec_ok, int64_t capacity_sum, int grid_override,
                         cudaStream_t st, int pipeline, int threads, int ctas_per_sm)
{
    // the grid is sized from the capacities (counts live on the device); idle
    // CTAs exit after reading the counts
    if constexpr (sizeof(T) == 4) {
        // the default: bulk copies, 15 consumer warps + the producer (16 warps, 4 per
        // scheduler), 2 stages of 1920-particle tiles: the fastest of 7 .. 18 consumer
        // warps and 2 .. 4 stages measured on GB300
        const bool dflt = pipeline == QED_EVOLVE_DEFAULT && threads == 0 && ctas_per_sm == 0;
        if (vec_ok && (pipeline == QED_EVOLVE_BULK || dflt) && grid_override <= 0) {
            if (dflt) return launch_bulk<15, 2, 1, MAXSEG>(a, capacity_sum, st);
            if (threads == 512) return launch_bulk<16, 2, 1, MAXSEG>(a, capacity_sum, st);
            if (ctas_per_sm == 2) return launch_bulk<8, 2, 2, MAXSEG>(a, capacity_sum, st);
            return launch_bulk<8, 4, 1, MAXSEG>(a, capacity_sum, st);
        }
    }
    if (vec_ok) {
        constexpr int V = sizeof(T) == 4 ? 4 : 2;
        if (sizeof(T) == 4 && ctas_per_sm != 3) {  // 64 registers: 32 warps per SM (the faster)
            const int g = grid_override > 0 ? grid_override : evolve_grid<T, V, MAXSEG, 4>(capacity_sum);
            evolve_kernel<T, V, MAXSEG, 4><<<g, kEvolveThreads, 0, st>>>(a);
        } else {
            const int g = grid_override > 0 ? grid_override : evolve_grid<T, V, MAXSEG>(capacity_sum);
            evolve_kernel<T, V, MAXSEG><<<g, kEvolveThreads, 0, st>>>(a);
        }
    } else {
        const int g = grid_override > 0 ? grid_override : evolve_grid<T, 1, MAXSEG>(capacity_sum);
        evolve_kernel<T, 1, MAXSEG><<<g, kEvolveThreads, 0, st>>>(a);
    }
    QED_LAUNCH_CHECK();
    return QED_OK;
}

template qed_status launch_evolve<float, 4>(const EvolveArgs<float, 4> &, bool, int64_t, int, cudaStream_t, int, int,
                                           int);
template qed_status launch_evolve<double, 4>(const EvolveArgs<double, 4> &, bool, int64_t, int, cudaStream_t, int,
                                            int, int);

static bool al16(const void *p) { return p == nullptr || ((uintptr_t)p & 15u) == 0; }

template <typename T>
bool fill_seg(EvolveSeg<T> &g, const qed_species *sp, int proc, const qed_fire_list *fire)
{
    g.px = (const T *)sp->px, g.py = (const T *)sp->py, g.pz = (const T *)sp->pz;
    g.ex = (const T *)sp->ex, g.ey = (const T *)sp->ey, g.ez = (const T *)sp->ez;
    g.bx = (const T *)sp->bx, g.by = (const T *)sp->by, g.bz = (const T *)sp->bz;
    g.tau = (T *)sp->tau;
    g.tau_c = (T *)sp->tau_c;
    g.count = sp->d_count;
    g.capacity = sp->capacity;
    g.fire_idx = fire->idx;
    g.fire_chi = fire->chi;
    g.fire_count = (unsigned long long *)fire->d_count;
    g.fire_cap = fire->capacity;
    g.proc = proc;
    const void *ps[] = {sp->px, sp->py, sp->pz, sp->ex, sp->ey, sp->ez, sp->bx, sp->by, sp->bz, sp->tau};
    bool ok = true;
    for (const void *p : ps) ok = ok && al16(p);
    if (sizeof(T) == 4) ok = ok && al16(sp->tau_c);
    return ok;
}

template bool fill_seg<float>(EvolveSeg<float> &, const qed_species *, int, const qed_fire_list *);
template bool fill_seg<double>(EvolveSeg<double> &, const qed_species *, int, const qed_fire_list *);

qed_status check_fire(const qed_fire_list *f, const char *name)
{
    if (!f) QED_FAIL(QED_ERR_INVALID_ARG, "%s: fire list is NULL", name);
    if (!f->idx || !f->chi || !f->d_count) QED_FAIL(QED_ERR_INVALID_ARG, "%s: fire list array is NULL", name);
    if (f->capacity < 0) QED_FAIL(QED_ERR_INVALID_ARG, "%s: negative fire-list capacity", name);
    return QED_OK;
}

// ---------------------------------------------------------------------------
// optical-depth initialisation: tau = -ln U(seed, (id, step, 2))
// ---------------------------------------------------------------------------
template <typename T>
__global__ void init_tau_kernel(T *tau, T *tau_c, const uint64_t *id, const int64_t *count, int64_t capacity,
                                uint64_t seed, int64_t step)
{
    int64_t n = *count;
    n = n < 0 ? 0 : (n > capacity ? capacity : n);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        store_tau<T>(tau, tau_c, i, tau_draw(seed, id[i], step, kTauInit));
}

}  // namespace qed

using namespace qed;

extern "C" qed_status qed_init_optical_depth(const qed_species *sp, qed_precision prec, uint64_t seed, int64_t step,
                                             void *stream)
{
    clear_error();
    qed_status s = check_species(sp, "species", prec);
    if (s) return s;
    cudaStream_t st = as_stream(stream);
    const int g = prec == QED_F32 ? resident_grid<init_tau_kernel<float>>(256, 0, sp->capacity)
                                  : resident_grid<init_tau_kernel<double>>(256, 0, sp->capacity);
    if (prec == QED_F32)
        init_tau_kernel<float><<<g, 256, 0, st>>>((float *)sp->tau, (float *)sp->tau_c, sp->id, sp->d_count,
                                                  sp->capacity, seed, step);
    else
        init_tau_kernel<double><<<g, 256, 0, st>>>((double *)sp->tau, nullptr, sp->id, sp->d_count, sp->capacity,
                                                   seed, step);
    QED_LAUNCH_CHECK();
    return QED_OK;
}

template <typename T>
static qed_status evolve_one_species(const qed_tables *t, qed_process proc, const qed_species *sp, double dt,
                                     const qed_fire_list *fire, int64_t *d_stats, cudaStream_t st)
{
    EvolveArgs<T, 4> a;
    memset(&a, 0, sizeof(a));
    a.n_seg = 1;
    a.dt = (T)dt;
    a.tab = make_view<T>(t);
    a.stats = (long long *)d_stats;
    const bool vec = fill_seg<T>(a.seg[0], sp, (int)proc, fire);
    QED_CUDA_TRY(cudaMemsetAsync(fire->d_count, 0, sizeof(int64_t), st));
    qed_status s = launch_evolve<T, 4>(a, vec, sp->capacity, 0, st);
    if (s) return s;
    clamp_fire_counts<<<1, 32, 0, st>>>((unsigned long long *)fire->d_count, fire->capacity, nullptr, 0, nullptr, 0);
    QED_LAUNCH_CHECK();
    return QED_OK;
}

extern "C" qed_status qed_evolve_optical_depth(const qed_tables *t, qed_process proc, const qed_species *sp,
                                               double dt, qed_precision prec, const qed_fire_list *fire,
                                               int64_t *d_stats, void *stream)
{
    clear_error();
    qed_status s;
    if ((s = check_tables(t))) return s;
    if ((s = check_species(sp, "species", prec))) return s;
    if ((s = check_fire(fire, "fire"))) return s;
    if (proc != QED_PROC_QS && proc != QED_PROC_BW) QED_FAIL(QED_ERR_INVALID_ARG, "bad process %d", (int)proc);
    if (!std::isfinite(dt) || dt < 0) QED_FAIL(QED_ERR_INVALID_ARG, "dt must be finite and >= 0");
    cudaStream_t st = as_stream(stream);
    return prec == QED_F32 ? evolve_one_species<float>(t, proc, sp, dt, fire, d_stats, st)
                           : evolve_one_species<double>(t, proc, sp, dt, fire, d_stats, st);
}
