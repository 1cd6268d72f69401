// events.cu -- the event kernels of the substep: quantum-synchrotron photon
// emission (§2.2, §3.2) and Breit-Wheeler pair production (§2.1, §3.1) for the
// particles in a firing list, and the fused substep entry point.
//
// Each warp takes 32 consecutive firing-list entries (all lanes stay in the
// loop, so ballots use the full mask).  Secondaries are appended with one
// atomic per warp on the destination's device count; a destination that is
// full leaves the event unexecuted (the parent keeps tau < 0 and fires again on
// the next step) and is counted in QED_STAT_DROPPED_CAPACITY.
#include "evolve.cuh"
#include "physics.cuh"

namespace qed {

template <typename T>
struct SpeciesPtrs {
    T *px, *py, *pz, *ex, *ey, *ez, *bx, *by, *bz, *tau, *tau_c, *w;
    uint64_t *id;
    unsigned long long *count;
    int64_t cap;
};

template <typename T>
static SpeciesPtrs<T> ptrs(const qed_species *s)
{
    SpeciesPtrs<T> p;
    p.px = (T *)s->px, p.py = (T *)s->py, p.pz = (T *)s->pz;
    p.ex = (T *)s->ex, p.ey = (T *)s->ey, p.ez = (T *)s->ez;
    p.bx = (T *)s->bx, p.by = (T *)s->by, p.bz = (T *)s->bz;
    p.tau = (T *)s->tau, p.tau_c = (T *)s->tau_c, p.w = (T *)s->weight;
    p.id = s->id;
    p.count = (unsigned long long *)s->d_count;
    p.cap = s->capacity;
    return p;
}

template <typename T>
struct EventArgs {
    SpeciesPtrs<T> parent, out0, out1;  // QS: out0 = photons; BW: out0 = electrons, out1 = positrons
    const int64_t *fire_idx;
    const double *fire_chi;
    const int64_t *fire_count;
    int64_t fire_cap;
    Table2D<T> tab;
    uint64_t seed;
    int64_t step;
    double threshold;
    long long *stats;
};

template <typename T>
__device__ __forceinline__ void write_particle(const SpeciesPtrs<T> &d, int64_t k, T px, T py, T pz, T ex, T ey,
                                               T ez, T bx, T by, T bz, T w, uint64_t id, double tau)
{
    d.px[k] = px, d.py[k] = py, d.pz[k] = pz;
    d.ex[k] = ex, d.ey[k] = ey, d.ez[k] = ez;
    d.bx[k] = bx, d.by[k] = by, d.bz[k] = bz;
    d.w[k] = w;
    d.id[k] = id;
    store_tau<T>(d.tau, d.tau_c, k, tau);
}

// placeholder written into a slot reserved for an event that could not run
template <typename T>
__device__ __forceinline__ void write_dead(const SpeciesPtrs<T> &d, int64_t k)
{
    write_particle<T>(d, k, T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), ~0ull,
                      (double)INFINITY);
}

__device__ __forceinline__ int64_t fire_n(const int64_t *c, int64_t cap)
{
    int64_t n = *c;
    return n < 0 ? 0 : (n > cap ? cap : n);
}

// ---------------------------------------------------------------------------
// photon emission
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) qs_event_kernel(const __grid_constant__ EventArgs<T> a)
{
    const int64_t nf = fire_n(a.fire_count, a.fire_cap);
    const unsigned lane = threadIdx.x & 31u;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int n_exec = 0, n_kept = 0, n_disc = 0, n_drop = 0;
    const SpeciesPtrs<T> &P = a.parent, &G = a.out0;

    for (int64_t base = warp * 32; base < nf; base += nwarp * 32) {
        const int64_t k = base + lane;
        const int64_t i0 = k < nf ? a.fire_idx[k] : -1;
        const bool valid = i0 >= 0 && i0 < P.cap;  // entries outside the parent are ignored
        const int64_t i = valid ? i0 : 0;
        const T chi = valid ? (T)a.fire_chi[k] : T(0);
        const T px = valid ? P.px[i] : T(0), py = valid ? P.py[i] : T(0), pz = valid ? P.pz[i] : T(1);
        const uint64_t pid = valid ? P.id[i] : 0;

        const U4 w = draw(a.seed, pid, a.step, kSample);
        const T r = sample_uniform<T>(uniform53(w.x, w.y));
        const T xi = valid ? qs_sample_xi<T>(a.tab, chi, r) : T(0);

        const T p2 = px * px + py * py + pz * pz;
        const T pm = d_sqrt(p2);
        const T gamma = d_sqrt(T(1) + p2);
        const T gg = (gamma - T(1)) * xi;  // photon energy (§2.2)
        const T g1 = gamma - gg;            // lepton energy after emission
        const T q = (g1 - T(1)) * (g1 + T(1));
        const T pn = d_sqrt(q > T(0) ? q : T(0));
        const T inv = pm > T(0) ? T(1) / pm : T(0);
        const T nx = px * inv, ny = py * inv, nz = pz * inv;

        const bool keep = valid && (double)gg >= a.threshold;
        const long long slot = warp_reserve(G.count, keep);
        const bool room = !keep || slot < G.cap;
        const bool exec = valid && room;
        n_drop += (valid && !room) ? 1 : 0;
        if (keep && room) {
            const U4 cid = draw(a.seed, pid, a.step, kChildId);
            const uint64_t child = ((uint64_t)cid.y << 32) | cid.x;
            write_particle<T>(G, slot, gg * nx, gg * ny, gg * nz, P.ex[i], P.ey[i], P.ez[i], P.bx[i], P.by[i],
                              P.bz[i], P.w[i], child, tau_draw(a.seed, child, a.step, kTauInit));
        }
        if (exec) {
            P.px[i] = pn * nx, P.py[i] = pn * ny, P.pz[i] = pn * nz;
            store_tau<T>(P.tau, P.tau_c, i, tau_draw(a.seed, pid, a.step, kTauReset));
        }
        n_exec += exec ? 1 : 0;
        n_kept += (keep && room) ? 1 : 0;
        n_disc += (exec && !keep) ? 1 : 0;
    }
    if (a.stats) {
        warp_count(a.stats + QED_STAT_QS_EVENTS, n_exec);
        warp_count(a.stats + QED_STAT_PHOTONS_KEPT, n_kept);
        warp_count(a.stats + QED_STAT_PHOTONS_DISCARDED, n_disc);
        warp_count(a.stats + QED_STAT_DROPPED_CAPACITY, n_drop);
    }
}

// ---------------------------------------------------------------------------
// pair production
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) bw_event_kernel(const __grid_constant__ EventArgs<T> a)
{
    const int64_t nf = fire_n(a.fire_count, a.fire_cap);
    const unsigned lane = threadIdx.x & 31u;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarp = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int n_exec = 0, n_pairs = 0, n_nopair = 0, n_drop = 0;
    const SpeciesPtrs<T> &P = a.parent, &E = a.out0, &Q = a.out1;

    for (int64_t base = warp * 32; base < nf; base += nwarp * 32) {
        const int64_t k = base + lane;
        const int64_t i0 = k < nf ? a.fire_idx[k] : -1;
        const bool valid = i0 >= 0 && i0 < P.cap;  // entries outside the parent are ignored
        const int64_t i = valid ? i0 : 0;
        const T chi = valid ? (T)a.fire_chi[k] : T(0);
        const T px = valid ? P.px[i] : T(0), py = valid ? P.py[i] : T(0), pz = valid ? P.pz[i] : T(1);
        const uint64_t pid = valid ? P.id[i] : 0;

        const U4 w = draw(a.seed, pid, a.step, kSample);
        bool electron = true;
        const T xs = valid ? bw_sample_xi<T>(a.tab, chi, uniform53(w.x, w.y), electron) : T(0);
        const T xm = electron ? xs : T(1) - xs;
        const T xp = electron ? T(1) - xs : xs;

        const T gg = d_sqrt(px * px + py * py + pz * pz);  // photon energy
        const bool pair = valid && gg > T(2);                // below 2 m_e c^2 no pair
        const T inv = gg > T(0) ? T(1) / gg : T(0);
        const T nx = px * inv, ny = py * inv, nz = pz * inv;
        const T km = (gg - T(2)) * xm, kp = (gg - T(2)) * xp;  // kinetic energies (§2.1)
        const T pmm = d_sqrt(km * (km + T(2))), pmp = d_sqrt(kp * (kp + T(2)));

        const long long se = warp_reserve(E.count, pair);
        const long long sq = warp_reserve(Q.count, pair);
        const bool ok_e = se < E.cap, ok_q = sq < Q.cap;
        const bool room = !pair || (ok_e && ok_q);
        const bool exec = valid && room;
        if (pair && !room) {
            ++n_drop;
            if (ok_e) write_dead<T>(E, se);
            if (ok_q) write_dead<T>(Q, sq);
        }
        if (pair && room) {
            const U4 cid = draw(a.seed, pid, a.step, kChildId);
            const uint64_t ide = ((uint64_t)cid.y << 32) | cid.x;
            const uint64_t idp = ((uint64_t)cid.w << 32) | cid.z;
            const T ex = P.ex[i], ey = P.ey[i], ez = P.ez[i], bx = P.bx[i], by = P.by[i], bz = P.bz[i], wt = P.w[i];
            write_particle<T>(E, se, pmm * nx, pmm * ny, pmm * nz, ex, ey, ez, bx, by, bz, wt, ide,
                              tau_draw(a.seed, ide, a.step, kTauInit));
            write_particle<T>(Q, sq, pmp * nx, pmp * ny, pmp * nz, ex, ey, ez, bx, by, bz, wt, idp,
                              tau_draw(a.seed, idp, a.step, kTauInit));
            // the photon is removed
            P.w[i] = T(0);
            P.tau[i] = T(INFINITY);
            if (sizeof(T) == 4) P.tau_c[i] = T(0);
        }
        if (valid && !pair) store_tau<T>(P.tau, P.tau_c, i, tau_draw(a.seed, pid, a.step, kTauReset));
        n_exec += exec ? 1 : 0;
        n_pairs += (pair && room) ? 1 : 0;
        n_nopair += (valid && !pair) ? 1 : 0;
    }
    if (a.stats) {
        warp_count(a.stats + QED_STAT_BW_EVENTS, n_exec);
        warp_count(a.stats + QED_STAT_PAIRS, n_pairs);
        warp_count(a.stats + QED_STAT_BW_NO_PAIR, n_nopair);
        warp_count(a.stats + QED_STAT_DROPPED_CAPACITY, n_drop);
    }
}

// keep every device count within its capacity after reservations overshoot
__global__ void clamp_counts(unsigned long long *c0, int64_t cap0, unsigned long long *c1, int64_t cap1)
{
    if (threadIdx.x == 0) {
        if (c0 && *c0 > (unsigned long long)cap0) *c0 = cap0;
        if (c1 && *c1 > (unsigned long long)cap1) *c1 = cap1;
    }
}

__global__ void zero3(int64_t *a, int64_t *b, int64_t *c)
{
    if (threadIdx.x == 0) *a = 0, *b = 0, *c = 0;
}

__device__ __forceinline__ void clamp1(unsigned long long *c, int64_t cap)
{
    if (c && *c > (unsigned long long)cap) *c = cap;
}

__global__ void clamp_all(unsigned long long *s0, int64_t c0, unsigned long long *s1, int64_t c1,
                          unsigned long long *s2, int64_t c2, unsigned long long *f0, int64_t d0,
                          unsigned long long *f1, int64_t d1, unsigned long long *f2, int64_t d2)
{
    if (threadIdx.x == 0) {
        clamp1(s0, c0), clamp1(s1, c1), clamp1(s2, c2), clamp1(f0, d0), clamp1(f1, d1), clamp1(f2, d2);
    }
}

static int event_grid(int64_t fire_cap)
{
    int64_t warps = (fire_cap + 31) / 32;
    int64_t blocks = (warps + 7) / 8;
    const int64_t cap = (int64_t)sm_count() * 4;
    blocks = blocks < 1 ? 1 : (blocks > cap ? cap : blocks);
    return (int)blocks;
}

template <typename T>
static qed_status launch_photons(const qed_tables *t, const qed_species *lep, const qed_species *ph,
                                 const qed_fire_list *fire, uint64_t seed, int64_t step, const qed_substep_opts *o,
                                 cudaStream_t st, bool clamp = true)
{
    EventArgs<T> a;
    memset(&a, 0, sizeof(a));
    a.parent = ptrs<T>(lep);
    a.out0 = ptrs<T>(ph);
    a.fire_idx = fire->idx;
    a.fire_chi = fire->chi;
    a.fire_count = fire->d_count;
    a.fire_cap = fire->capacity;
    a.tab = make_view<T>(t).qs_P;
    a.seed = seed;
    a.step = step;
    a.threshold = o ? o->photon_threshold : 0.0;
    a.stats = o ? (long long *)o->d_stats : nullptr;
    qs_event_kernel<T><<<event_grid(fire->capacity), 256, 0, st>>>(a);
    QED_LAUNCH_CHECK();
    if (clamp) {
        clamp_counts<<<1, 32, 0, st>>>(a.out0.count, a.out0.cap, nullptr, 0);
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
    a.parent = ptrs<T>(ph);
    a.out0 = ptrs<T>(el);
    a.out1 = ptrs<T>(po);
    a.fire_idx = fire->idx;
    a.fire_chi = fire->chi;
    a.fire_count = fire->d_count;
    a.fire_cap = fire->capacity;
    a.tab = make_view<T>(t).bw_P;
    a.seed = seed;
    a.step = step;
    a.stats = o ? (long long *)o->d_stats : nullptr;
    bw_event_kernel<T><<<event_grid(fire->capacity), 256, 0, st>>>(a);
    QED_LAUNCH_CHECK();
    if (clamp) {
        clamp_counts<<<1, 32, 0, st>>>(a.out0.count, a.out0.cap, a.out1.count, a.out1.cap);
        QED_LAUNCH_CHECK();
    }
    return QED_OK;
}

static qed_status check_opts(const qed_substep_opts *o)
{
    if (o && o->sampler != 0) QED_FAIL(QED_ERR_UNSUPPORTED, "sampler %d is served by the qed_mlp entry points", o->sampler);
    if (o && !(o->photon_threshold >= 0.0)) QED_FAIL(QED_ERR_INVALID_ARG, "photon_threshold must be >= 0");
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
    bool vec = fill_seg<T>(a.seg[0], e, QED_PROC_QS, &fire[0]);
    vec = fill_seg<T>(a.seg[1], p, QED_PROC_QS, &fire[1]) && vec;
    vec = fill_seg<T>(a.seg[2], g, QED_PROC_BW, &fire[2]) && vec;
    zero3<<<1, 32, 0, st>>>(fire[0].d_count, fire[1].d_count, fire[2].d_count);
    QED_LAUNCH_CHECK();
    if (o && o->evolve_begin) QED_CUDA_TRY(cudaEventRecord((cudaEvent_t)o->evolve_begin, st));
    qed_status s = launch_evolve<T, 4>(a, vec, e->capacity + p->capacity + g->capacity, 0, st);
    if (s) return s;
    if (o && o->evolve_end) QED_CUDA_TRY(cudaEventRecord((cudaEvent_t)o->evolve_end, st));
    // the event kernels clamp the firing counts on read and the species counts
    // after their appends
    if ((s = launch_pairs<T>(t, g, e, p, &fire[2], seed, step, o, st, false))) return s;
    if ((s = launch_photons<T>(t, e, g, &fire[0], seed, step, o, st, false))) return s;
    if ((s = launch_photons<T>(t, p, g, &fire[1], seed, step, o, st, false))) return s;
    clamp_all<<<1, 32, 0, st>>>(ptrs<T>(e).count, e->capacity, ptrs<T>(p).count, p->capacity, ptrs<T>(g).count,
                                g->capacity, (unsigned long long *)fire[0].d_count, fire[0].capacity,
                                (unsigned long long *)fire[1].d_count, fire[1].capacity,
                                (unsigned long long *)fire[2].d_count, fire[2].capacity);
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
