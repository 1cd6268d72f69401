// events.cu -- the event kernels of the substep for one firing list each:
// quantum-synchrotron photon emission (§2.2, §3.2) and Breit-Wheeler pair
// production (§2.1, §3.1), one kernel for the three lists of a substep, and the
// fused three-species substep entry point.
// The per-warp routines are in events.cuh (shared with the batched kernels).
#include <cmath>

#include "events.cuh"
#include "evolve.cuh"

namespace qed {

template <typename T>
struct EventArgs {
    EventSeg<T> seg;
    EventCommon<T> com;
};

template <typename T, bool MLP>
__global__ void __launch_bounds__(256) qs_event_kernel(const __grid_constant__ EventArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    InferSmem &S = *reinterpret_cast<InferSmem *>(smem_raw);
    if constexpr (MLP) {
        mlp_stage(S.net, a.com.mlpv.w);
        __syncthreads();
    }
    const int64_t nf = fire_n(a.seg.fire_count, a.seg.fire_cap);
    const int64_t step = event_step(a.com.d_step, a.com.step);
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    EventCounts k;
    for (int64_t base = warp * 32; base < nf; base += nwarp * 32)
        qs_event_chunk<T, MLP>(a.seg, a.com, step, base, nf, S, k);
    flush_counts(a.com.stats, k, true);
}

template <typename T, bool MLP>
__global__ void __launch_bounds__(256) bw_event_kernel(const __grid_constant__ EventArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    InferSmem &S = *reinterpret_cast<InferSmem *>(smem_raw);
    if constexpr (MLP) {
        mlp_stage(S.net, a.com.mlpv.w);
        __syncthreads();
    }
    const int64_t nf = fire_n(a.seg.fire_count, a.seg.fire_cap);
    const int64_t step = event_step(a.com.d_step, a.com.step);
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    EventCounts k;
    for (int64_t base = warp * 32; base < nf; base += nwarp * 32)
        bw_event_chunk<T, MLP>(a.seg, a.com, step, base, nf, S, k);
    flush_counts(a.com.stats, k, false);
}

// The three firing lists of one substep in one launch (table sampler):
// photon emission of the electrons and of the positrons, pair production of
// the photons.  They touch disjoint particles (each reads and updates its own
// parents below the pre-step counts and appends to another species), so their
// chunks of 32 entries run side by side; the chunk index runs over the three
// lists one after the other.
template <typename T>
struct Events3Args {
    EventSeg<T> seg[3];  // electrons -> photons, positrons -> photons, photons -> pairs
    EventCommon<T> qs, bw;
};

template <typename T>
__global__ void __launch_bounds__(256) events3_kernel(const __grid_constant__ Events3Args<T> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    InferSmem &S = *reinterpret_cast<InferSmem *>(smem_raw);  // (not touched without the learned sampler)
    int64_t nf[3], c1, c2, c3;
#pragma unroll
    for (int k = 0; k < 3; ++k) nf[k] = fire_n(a.seg[k].fire_count, a.seg[k].fire_cap);
    c1 = (nf[0] + 31) / 32;
    c2 = c1 + (nf[1] + 31) / 32;
    c3 = c2 + (nf[2] + 31) / 32;
    const int64_t step = event_step(a.qs.d_step, a.qs.step);
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    EventCounts kq, kb;
    for (int64_t c = warp; c < c3; c += nwarp) {
        if (c < c1)
            qs_event_chunk<T, false>(a.seg[0], a.qs, step, c * 32, nf[0], S, kq);
        else if (c < c2)
            qs_event_chunk<T, false>(a.seg[1], a.qs, step, (c - c1) * 32, nf[1], S, kq);
        else
            bw_event_chunk<T, false>(a.seg[2], a.bw, step, (c - c2) * 32, nf[2], S, kb);
    }
    flush_counts(a.qs.stats, kq, true);
    flush_counts(a.bw.stats, kb, false);
}

__global__ void zero3(int64_t *a, int64_t *b, int64_t *c)
{
    if (threadIdx.x == 0) *a = 0, *b = 0, *c = 0;
}

__device__ __forceinline__ void clamp1(unsigned long long *c, int64_t cap)
{
    if (c && *c > (unsigned long long)cap) *c = cap;
}

// keep the device counts within their capacities after the reservations of the
// event kernels overshot, and advance the device step counter if there is one
__global__ void clamp_all(unsigned long long *s0, int64_t c0, unsigned long long *s1, int64_t c1,
                          unsigned long long *s2, int64_t c2, unsigned long long *f0, int64_t d0,
                          unsigned long long *f1, int64_t d1, unsigned long long *f2, int64_t d2, int64_t *step)
{
    if (threadIdx.x == 0) {
        clamp1(s0, c0), clamp1(s1, c1), clamp1(s2, c2), clamp1(f0, d0), clamp1(f1, d1), clamp1(f2, d2);
        if (step) *step += 1;
    }
}

// CTAs of 256 threads for a firing list of fire_cap entries (a warp per chunk
// of 32), at most as many as stay resident: every CTA strides over the chunks,
// so a CTA that has to wait for a second wave only lengthens the launch
template <auto Kernel>
static int event_grid(size_t dyn, int64_t fire_cap)
{
    static int per_sm = 0;  // one per kernel
    if (per_sm == 0) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, Kernel, 256, dyn);
        if (per_sm <= 0) per_sm = 1;
    }
    int64_t warps = (fire_cap + 31) / 32;
    int64_t blocks = (warps + 7) / 8;
    const int64_t cap = (int64_t)sm_count() * per_sm;
    blocks = blocks < 1 ? 1 : (blocks > cap ? cap : blocks);
    return (int)blocks;
}

template <typename T>
EventCommon<T> event_common(const qed_tables *t, int proc, uint64_t seed, int64_t step, const qed_substep_opts *o)
{
    EventCommon<T> c;
    memset(&c, 0, sizeof(c));
    const TablesView<T> v = make_view<T>(t);
    c.tab = proc == QED_PROC_QS ? v.qs_P : v.bw_P;
    c.seed = seed;
    c.step = step;
    c.d_step = o ? o->d_step : nullptr;
    c.threshold = o ? o->photon_threshold : 0.0;
    c.threshold_f = (float)c.threshold;
    if ((double)c.threshold_f < c.threshold) c.threshold_f = std::nextafter(c.threshold_f, INFINITY);
    c.stats = o ? (long long *)o->d_stats : nullptr;
    c.copy_fields = 1;
    if (o && o->sampler == 1) c.mlpv = mlp_view((const qed_mlp *)o->mlp, proc);
    return c;
}

template EventCommon<float> event_common<float>(const qed_tables *, int, uint64_t, int64_t, const qed_substep_opts *);
template EventCommon<double> event_common<double>(const qed_tables *, int, uint64_t, int64_t,
                                                  const qed_substep_opts *);

template <typename K>
static qed_status allow_infer_smem(K kernel)
{
    QED_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(InferSmem)));
    return QED_OK;
}

template <typename T>
static qed_status launch_photons(const qed_tables *t, const qed_species *lep, const qed_species *ph,
                                 const qed_fire_list *fire, uint64_t seed, int64_t step, const qed_substep_opts *o,
                                 cudaStream_t st, bool clamp = true)
{
    EventArgs<T> a;
    memset(&a, 0, sizeof(a));
    a.seg.parent = ptrs<T>(lep);
    a.seg.out0 = ptrs<T>(ph);
    a.seg.fire_idx = fire->idx;
    a.seg.fire_chi = fire->chi;
    a.seg.fire_count = fire->d_count;
    a.seg.fire_cap = fire->capacity;
    a.com = event_common<T>(t, QED_PROC_QS, seed, step, o);
    if (o && o->sampler == 1) {
        static bool attr = false;
        if (!attr) {
            qed_status s = allow_infer_smem(qs_event_kernel<T, true>);
            if (s) return s;
            attr = true;
        }
        qs_event_kernel<T, true>
            <<<event_grid<qs_event_kernel<T, true>>(sizeof(InferSmem), fire->capacity), 256, sizeof(InferSmem), st>>>(
                a);
    } else {
        qs_event_kernel<T, false><<<event_grid<qs_event_kernel<T, false>>(0, fire->capacity), 256, 0, st>>>(a);
    }
    QED_LAUNCH_CHECK();
    if (clamp) {
        clamp_all<<<1, 32, 0, st>>>(a.seg.out0.count, a.seg.out0.cap, nullptr, 0, nullptr, 0, nullptr, 0, nullptr, 0,
                                    nullptr, 0, nullptr);
        QED_LAUNCH_CHECK();
    }
    return QED_OK;
}

template <typename T>
static qed_status launch_pairs(const qed_tables *t, const qed_species *ph, const qed_species *el,
                               const qed_species *po, const qed_fire_list *fire, uint64_t seed, int64_t step,
                               const qed_substep_opts *o, cudaStream_t st, bool clamp = true)
{
    EventArgs<T> a;
    memset(&a, 0, sizeof(a));
    a.seg.parent = ptrs<T>(ph);
    a.seg.out0 = ptrs<T>(el);
    a.seg.out1 = ptrs<T>(po);
    a.seg.fire_idx = fire->idx;
    a.seg.fire_chi = fire->chi;
    a.seg.fire_count = fire->d_count;
    a.seg.fire_cap = fire->capacity;
    a.com = event_common<T>(t, QED_PROC_BW, seed, step, o);
    if (o && o->sampler == 1) {
        static bool attr = false;
        if (!attr) {
            qed_status s = allow_infer_smem(bw_event_kernel<T, true>);
            if (s) return s;
            attr = true;
        }
        bw_event_kernel<T, true>
            <<<event_grid<bw_event_kernel<T, true>>(sizeof(InferSmem), fire->capacity), 256, sizeof(InferSmem), st>>>(
                a);
    } else {
        bw_event_kernel<T, false><<<event_grid<bw_event_kernel<T, false>>(0, fire->capacity), 256, 0, st>>>(a);
    }
    QED_LAUNCH_CHECK();
    if (clamp) {
        clamp_all<<<1, 32, 0, st>>>(a.seg.out0.count, a.seg.out0.cap, a.seg.out1.count, a.seg.out1.cap, nullptr, 0,
                                    nullptr, 0, nullptr, 0, nullptr, 0, nullptr);
        QED_LAUNCH_CHECK();
    }
    return QED_OK;
}

qed_status check_opts(const qed_substep_opts *o)
{
    if (o && o->sampler != 0 && o->sampler != 1) QED_FAIL(QED_ERR_INVALID_ARG, "unknown sampler %d", o->sampler);
    if (o && o->sampler == 1 && o->mlp == nullptr) QED_FAIL(QED_ERR_INVALID_ARG, "sampler 1 needs opts->mlp");
    if (o && !(o->photon_threshold >= 0.0)) QED_FAIL(QED_ERR_INVALID_ARG, "photon_threshold must be >= 0");
    if (o && !(o->qs_chi_cut >= 0.0 && o->bw_chi_cut >= 0.0))
        QED_FAIL(QED_ERR_INVALID_ARG, "qs_chi_cut and bw_chi_cut must be >= 0");
    if (o && (o->evolve_pipeline < QED_EVOLVE_DEFAULT || o->evolve_pipeline > QED_EVOLVE_BULK))
        QED_FAIL(QED_ERR_INVALID_ARG, "unknown evolve_pipeline %d", o->evolve_pipeline);
    return QED_OK;
}

template <typename T>
static qed_status substep_impl(const qed_tables *t, const qed_species *e, const qed_species *p,
                               const qed_species *g, double dt, uint64_t seed, int64_t step,
                               const qed_substep_opts *o, const qed_fire_list *fire, cudaStream_t st)
{
    EvolveArgs<T, 4> a;
    memset(&a, 0, sizeof(a));
    a.n_seg = 3;
    a.dt = (T)dt;
    a.tab = make_view<T>(t);
    a.stats = o ? (long long *)o->d_stats : nullptr;
    a.chi_cut[QED_PROC_QS] = o ? (T)o->qs_chi_cut : T(0);
    a.chi_cut[QED_PROC_BW] = o ? (T)o->bw_chi_cut : T(0);
    a.wait_cycles = o ? o->wait_limit_cycles : 0;
    bool vec = fill_seg<T>(a.seg[0], e, QED_PROC_QS, &fire[0]);
    vec = fill_seg<T>(a.seg[1], p, QED_PROC_QS, &fire[1]) && vec;
    vec = fill_seg<T>(a.seg[2], g, QED_PROC_BW, &fire[2]) && vec;
    zero3<<<1, 32, 0, st>>>(fire[0].d_count, fire[1].d_count, fire[2].d_count);
    QED_LAUNCH_CHECK();
    if (o && o->evolve_begin) QED_CUDA_TRY(cudaEventRecord((cudaEvent_t)o->evolve_begin, st));
    qed_status s = launch_evolve<T, 4>(a, vec, e->capacity + p->capacity + g->capacity, 0, st,
                                       o ? o->evolve_pipeline : 0, o ? o->evolve_threads : 0,
                                       o ? o->evolve_ctas_per_sm : 0);
    if (s) return s;
    if (o && o->evolve_end) QED_CUDA_TRY(cudaEventRecord((cudaEvent_t)o->evolve_end, st));
    // the event kernels clamp the firing counts on read and the species counts
    // after their appends
    if (o && o->sampler == 1) {
        if ((s = launch_pairs<T>(t, g, e, p, &fire[2], seed, step, o, st, false))) return s;
        if ((s = launch_photons<T>(t, e, g, &fire[0], seed, step, o, st, false))) return s;
        if ((s = launch_photons<T>(t, p, g, &fire[1], seed, step, o, st, false))) return s;
    } else {
        Events3Args<T> ea;
        memset(&ea, 0, sizeof(ea));
        const qed_species *par[3] = {e, p, g};
        for (int k = 0; k < 3; ++k) {
            EventSeg<T> &sg = ea.seg[k];
            sg.parent = ptrs<T>(par[k]);
            sg.fire_idx = fire[k].idx;
            sg.fire_chi = fire[k].chi;
            sg.fire_count = fire[k].d_count;
            sg.fire_cap = fire[k].capacity;
        }
        ea.seg[0].out0 = ea.seg[1].out0 = ptrs<T>(g);
        ea.seg[2].out0 = ptrs<T>(e);
        ea.seg[2].out1 = ptrs<T>(p);
        ea.qs = event_common<T>(t, QED_PROC_QS, seed, step, o);
        ea.bw = event_common<T>(t, QED_PROC_BW, seed, step, o);
        const int g3 = event_grid<events3_kernel<T>>(0, fire[0].capacity + fire[1].capacity + fire[2].capacity);
        events3_kernel<T><<<g3, 256, 0, st>>>(ea);
        QED_LAUNCH_CHECK();
    }
    clamp_all<<<1, 32, 0, st>>>(ptrs<T>(e).count, e->capacity, ptrs<T>(p).count, p->capacity, ptrs<T>(g).count,
                                g->capacity, (unsigned long long *)fire[0].d_count, fire[0].capacity,
                                (unsigned long long *)fire[1].d_count, fire[1].capacity,
                                (unsigned long long *)fire[2].d_count, fire[2].capacity, o ? o->d_step : nullptr);
    QED_LAUNCH_CHECK();
    return QED_OK;
}

}  // namespace qed

using namespace qed;

extern "C" qed_status qed_generate_photons(const qed_tables *t, const qed_species *leptons,
                                           const qed_species *photons, const qed_fire_list *fire, uint64_t seed,
                                           int64_t step, const qed_substep_opts *opts, qed_precision prec,
                                           void *stream)
{
    clear_error();
    qed_status s;
    if ((s = check_tables(t))) return s;
    if ((s = check_species(leptons, "leptons", prec))) return s;
    if ((s = check_species(photons, "photons", prec))) return s;
    if ((s = check_fire(fire, "fire"))) return s;
    if ((s = check_opts(opts))) return s;
    cudaStream_t st = as_stream(stream);
    return prec == QED_F32 ? launch_photons<float>(t, leptons, photons, fire, seed, step, opts, st)
                           : launch_photons<double>(t, leptons, photons, fire, seed, step, opts, st);
}

extern "C" qed_status qed_generate_pairs(const qed_tables *t, const qed_species *photons,
                                         const qed_species *electrons, const qed_species *positrons,
                                         const qed_fire_list *fire, uint64_t seed, int64_t step,
                                         const qed_substep_opts *opts, qed_precision prec, void *stream)
{
    clear_error();
    qed_status s;
    if ((s = check_tables(t))) return s;
    if ((s = check_species(photons, "photons", prec))) return s;
    if ((s = check_species(electrons, "electrons", prec))) return s;
    if ((s = check_species(positrons, "positrons", prec))) return s;
    if ((s = check_fire(fire, "fire"))) return s;
    if ((s = check_opts(opts))) return s;
    cudaStream_t st = as_stream(stream);
    return prec == QED_F32 ? launch_pairs<float>(t, photons, electrons, positrons, fire, seed, step, opts, st)
                           : launch_pairs<double>(t, photons, electrons, positrons, fire, seed, step, opts, st);
}

extern "C" qed_status qed_substep(const qed_tables *t, const qed_species *electrons, const qed_species *positrons,
                                  const qed_species *photons, double dt, uint64_t seed, int64_t step,
                                  const qed_substep_opts *opts, qed_precision prec, const qed_fire_list *fire,
                                  void *stream)
{
    clear_error();
    qed_status s;
    if ((s = check_tables(t))) return s;
    if ((s = check_species(electrons, "electrons", prec))) return s;
    if ((s = check_species(positrons, "positrons", prec))) return s;
    if ((s = check_species(photons, "photons", prec))) return s;
    if (!fire) QED_FAIL(QED_ERR_INVALID_ARG, "fire is NULL");
    for (int k = 0; k < 3; ++k)
        if ((s = check_fire(&fire[k], "fire"))) return s;
    if ((s = check_opts(opts))) return s;
    if (!std::isfinite(dt) || dt < 0) QED_FAIL(QED_ERR_INVALID_ARG, "dt must be finite and >= 0");
    cudaStream_t st = as_stream(stream);
    return prec == QED_F32 ? substep_impl<float>(t, electrons, positrons, photons, dt, seed, step, opts, fire, st)
                           : substep_impl<double>(t, electrons, positrons, photons, dt, seed, step, opts, fire, st);
}
