// fused.cu -- the cascade step's per-particle pass in one launch over every
// species of every patch: the plane wave's fields at the particle, the Boris
// push, and the optical-depth evolution with compaction of the firing
// particles, on the same registers.  x, y, z, p, tau (and tau_c) are read and
// written once: 64 B per particle-step in FP32, against 124 B for the separate
// push (which stores the fields) and evolution (which loads them again).  The
// arithmetic is the separate kernels' own (pusher.cuh, evolve_core.cuh), so
// the particles end with the same bits; only the field arrays are left alone
// unless asked for.
#include "evolve_core.cuh"
#include "pusher.cuh"

namespace qed {

template <typename T, int VEC>
__device__ __forceinline__ void load_or_zero(const T *p, int64_t i0, int64_t n, bool full, T (&v)[VEC])
{
    if (full) {
        load_vec<T, VEC>(p, i0, v);
    } else {
#pragma unroll
        for (int j = 0; j < VEC; ++j) v[j] = i0 + j < n ? p[i0 + j] : T(0);
    }
}

template <typename T, int VEC>
__device__ __forceinline__ void store_live(T *p, int64_t i0, int64_t n, bool full, const T (&v)[VEC])
{
    if (full) {
        store_vec<T, VEC>(p, i0, v);
    } else {
#pragma unroll
        for (int j = 0; j < VEC; ++j)
            if (i0 + j < n) p[i0 + j] = v[j];
    }
}

// FP32: two particles per thread, 4 CTAs of 256 per SM (64 registers), the
// fastest of VEC 1 / 2 / 4 x 2 .. 4 CTAs per SM measured on GB300
template <typename T, int VEC, int THREADS>
__global__ void __launch_bounds__(THREADS, sizeof(T) == 4 ? 4 : 2)
    push_evolve_kernel(const EvolveSeg<T> *__restrict__ segs, const PushSeg<T> *__restrict__ psegs, int n_seg,
                       TablesView<T> tab, WaveParams w, double t0, double dt_d, const int64_t *d_step, int64_t step,
                       T cut_qs, T cut_bw, long long *stats, int store_fields)
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
    const WaveT<T> wt = wave_at<T>(w, t0 + (double)(d_step ? *d_step : step) * dt_d);
    const T dt = (T)dt_d;
    int bad = 0;
    int s = 0;
    for (long long t = blockIdx.x; t < total; t += gridDim.x) {
        while (s_end[s] <= t) ++s;  // tiles ascend, so the segment (first s_end[s] > t) only moves forward
        const EvolveSeg<T> &sg = segs[s];
        const PushSeg<T> &pg = psegs[s];
        const int64_t n = s_n[s];
        const int64_t i0 = (t - (s ? s_end[s - 1] : 0)) * tile + (int64_t)threadIdx.x * VEC;
        const bool full = i0 + VEC <= n;
        T x[VEC], y[VEC], z[VEC], px[VEC], py[VEC], pz[VEC], tau[VEC], tc[VEC];
        load_or_zero<T, VEC>(pg.x, i0, n, full, x);
        load_or_zero<T, VEC>(pg.y, i0, n, full, y);
        load_or_zero<T, VEC>(pg.z, i0, n, full, z);
        load_or_zero<T, VEC>(pg.px, i0, n, full, px);
        load_or_zero<T, VEC>(pg.py, i0, n, full, py);
        load_or_zero<T, VEC>(pg.pz, i0, n, full, pz);
        load_or_zero<T, VEC>(sg.tau, i0, n, full, tau);
        if constexpr (sizeof(T) == 4) {
            load_or_zero<T, VEC>(sg.tau_c, i0, n, full, tc);
        } else {
#pragma unroll
            for (int j = 0; j < VEC; ++j) tc[j] = T(0);
        }
        // each particle from its fields to its firing decision in one go: the
        // fields of one particle are live at a time
        const T cut = sg.proc == QED_PROC_QS ? cut_qs : cut_bw;
        bool fire[VEC];
        T chi[VEC];
        int cnt = 0;
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
            T ex, ey, ez, bx, by, bz, vx, vy, vz;
            wave_fields<T>(wt, x[j], ex, ey, ez, bx, by, bz);
            boris_move<T>(pg.q, dt, ex, ey, ez, bx, by, bz, px[j], py[j], pz[j], vx, vy, vz);
            x[j] = x[j] + vx * dt;
            y[j] = y[j] + vy * dt;
            z[j] = z[j] + vz * dt;
            if (store_fields && i0 + j < n) {
                pg.ex[i0 + j] = ex, pg.ey[i0 + j] = ey, pg.ez[i0 + j] = ez;
                pg.bx[i0 + j] = bx, pg.by[i0 + j] = by, pg.bz[i0 + j] = bz;
            }
            T c = tc[j];
            fire[j] = evolve_one<T>(sg.proc, s_qs, s_bw, tab, px[j], py[j], pz[j], ex, ey, ez, bx, by, bz, dt, cut,
                                    tau[j], c, chi[j], bad);
            tc[j] = c;
            fire[j] = fire[j] && (i0 + j < n);
            cnt += fire[j] ? 1 : 0;
        }
        store_live<T, VEC>(pg.x, i0, n, full, x);
        store_live<T, VEC>(pg.y, i0, n, full, y);
        store_live<T, VEC>(pg.z, i0, n, full, z);
        if (pg.q != T(0)) {
            store_live<T, VEC>(pg.px, i0, n, full, px);
            store_live<T, VEC>(pg.py, i0, n, full, py);
            store_live<T, VEC>(pg.pz, i0, n, full, pz);
        }
        store_live<T, VEC>(sg.tau, i0, n, full, tau);
        if constexpr (sizeof(T) == 4) store_live<T, VEC>(sg.tau_c, i0, n, full, tc);
        compact_fire<T, VEC>(sg, i0, fire, chi, cnt, stats);
    }
    warp_count_err(stats ? stats + QED_STAT_NONFINITE : nullptr, bad, QED_EW_NONFINITE);
}

template <typename T, int VEC>
static qed_status launch_fused_impl(const EvolveSeg<T> *segs, const PushSeg<T> *psegs, int n_seg,
                                    const TablesView<T> &tab, const WaveParams &w, double t0, double dt,
                                    const int64_t *d_step, int64_t step, T cut_qs, T cut_bw, long long *stats,
                                    int store_fields, cudaStream_t st)
{
    constexpr int kThreads = 256;
    const size_t dyn = (size_t)n_seg * 2 * sizeof(long long);
    static bool attr = false;
    static int per_sm = 0;
    if (!attr) {
        QED_CUDA_TRY(cudaFuncSetAttribute(push_evolve_kernel<T, VEC, kThreads>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          3 * QED_MAX_PATCHES * 2 * (int)sizeof(long long)));
        QED_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, push_evolve_kernel<T, VEC, kThreads>,
                                                                   kThreads, dyn));
        if (per_sm < 1) per_sm = 1;
        attr = true;
    }
    push_evolve_kernel<T, VEC, kThreads><<<sm_count() * per_sm, kThreads, dyn, st>>>(
        segs, psegs, n_seg, tab, w, t0, dt, d_step, step, cut_qs, cut_bw, stats, store_fields);
    QED_LAUNCH_CHECK();
    return QED_OK;
}

template <typename T>
qed_status launch_push_evolve(const EvolveSeg<T> *d_segs, const void *d_push, int n_seg, const TablesView<T> &tab,
                              const WaveParams &w, double t0, double dt, const int64_t *d_step, int64_t step,
                              T cut_qs, T cut_bw, long long *stats, int store_fields, bool vec, cudaStream_t st)
{
    if (n_seg <= 0) return QED_OK;
    const PushSeg<T> *p = (const PushSeg<T> *)d_push;
    if (vec) {
        constexpr int V = 2;
        return launch_fused_impl<T, V>(d_segs, p, n_seg, tab, w, t0, dt, d_step, step, cut_qs, cut_bw, stats,
                                       store_fields, st);
    }
    return launch_fused_impl<T, 1>(d_segs, p, n_seg, tab, w, t0, dt, d_step, step, cut_qs, cut_bw, stats,
                                   store_fields, st);
}

template qed_status launch_push_evolve<float>(const EvolveSeg<float> *, const void *, int, const TablesView<float> &,
                                              const WaveParams &, double, double, const int64_t *, int64_t, float,
                                              float, long long *, int, bool, cudaStream_t);
template qed_status launch_push_evolve<double>(const EvolveSeg<double> *, const void *, int,
                                               const TablesView<double> &, const WaveParams &, double, double,
                                               const int64_t *, int64_t, double, double, long long *, int, bool,
                                               cudaStream_t);

}  // namespace qed
