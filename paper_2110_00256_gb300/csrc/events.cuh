// events.cuh -- per-warp event routines shared by the single-call and the
// batched (many patches) event kernels: quantum-synchrotron photon emission
// (§2.2, §3.2) and Breit-Wheeler pair production (§2.1, §3.1).
//
// A warp takes 32 consecutive entries of one firing list (all lanes stay
// together, so ballots use the full mask).  Secondaries are appended with one
// atomic per warp on the destination's device count; a destination that is
// full leaves the event unexecuted (the parent keeps tau < 0 and fires again on
// the next step) and is counted in QED_STAT_DROPPED_CAPACITY.
#pragma once

#include "mlp.cuh"
#include "physics.cuh"

namespace qed {

template <typename T>
struct SpeciesPtrs {
    T *px, *py, *pz, *ex, *ey, *ez, *bx, *by, *bz, *tau, *tau_c, *w;
    T *x, *y, *z;  // positions, may be null
    uint64_t *id;
    unsigned long long *count;
    int64_t cap;
};

template <typename T>
inline SpeciesPtrs<T> ptrs(const qed_species *s)
{
    SpeciesPtrs<T> p;
    p.px = (T *)s->px, p.py = (T *)s->py, p.pz = (T *)s->pz;
    p.ex = (T *)s->ex, p.ey = (T *)s->ey, p.ez = (T *)s->ez;
    p.bx = (T *)s->bx, p.by = (T *)s->by, p.bz = (T *)s->bz;
    p.tau = (T *)s->tau, p.tau_c = (T *)s->tau_c, p.w = (T *)s->weight;
    p.x = (T *)s->x, p.y = (T *)s->y, p.z = (T *)s->z;
    p.id = s->id;
    p.count = (unsigned long long *)s->d_count;
    p.cap = s->capacity;
    return p;
}

// one firing list with its parent species and destination species
template <typename T>
struct EventSeg {
    SpeciesPtrs<T> parent, out0, out1;  // QS: out0 = photons; BW: out0 = electrons, out1 = positrons
    const int64_t *fire_idx;
    const double *fire_chi;
    const int64_t *fire_count;
    int64_t fire_cap;
};

template <typename T>
struct EventCommon {
    Table2D<T> tab;
    MlpView mlpv;             // used when the kernel is instantiated with the learned sampler
    uint64_t seed;
    int64_t step;
    const int64_t *d_step;    // if set, the step is read from here
    double threshold;
    float threshold_f;        // the smallest float >= threshold: gg >= threshold_f iff (double)gg >= threshold
    long long *stats;
    int copy_fields;          // 0: products get no field values (the caller computes them, see qed_push_substep_batched)
};

struct EventCounts {
    int exec = 0, kept = 0, disc = 0, drop = 0, pairs = 0, nopair = 0;
};

template <typename T>
__device__ __forceinline__ void write_particle(const SpeciesPtrs<T> &d, int64_t k, T px, T py, T pz, T ex, T ey,
                                               T ez, T bx, T by, T bz, T w, uint64_t id, double tau,
                                               bool fields = true)
{
    d.px[k] = px, d.py[k] = py, d.pz[k] = pz;
    if (fields) {
        d.ex[k] = ex, d.ey[k] = ey, d.ez[k] = ez;
        d.bx[k] = bx, d.by[k] = by, d.bz[k] = bz;
    }
    d.w[k] = w;
    d.id[k] = id;
    store_tau<T>(d.tau, d.tau_c, k, tau);
}

// the product sits where its parent is
template <typename T>
__device__ __forceinline__ void copy_position(const SpeciesPtrs<T> &d, int64_t k, const SpeciesPtrs<T> &p, int64_t i)
{
    if (d.x && p.x) d.x[k] = p.x[i], d.y[k] = p.y[i], d.z[k] = p.z[i];
}

// placeholder written into a slot reserved for an event that could not run
template <typename T>
__device__ __forceinline__ void write_dead(const SpeciesPtrs<T> &d, int64_t k)
{
    write_particle<T>(d, k, T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), T(0), ~0ull,
                      (double)INFINITY);
    if (d.x) d.x[k] = T(0), d.y[k] = T(0), d.z[k] = T(0);
}

__device__ __forceinline__ int64_t fire_n(const int64_t *c, int64_t cap)
{
    int64_t n = *c;
    return n < 0 ? 0 : (n > cap ? cap : n);
}

__device__ __forceinline__ int64_t event_step(const int64_t *d_step, int64_t step) { return d_step ? *d_step : step; }

// photon emission for entries [base, base + 32) of a firing list of nf entries
template <typename T, bool MLP>
__device__ __forceinline__ void qs_event_chunk(const EventSeg<T> &g, const EventCommon<T> &c, int64_t step,
                                               int64_t base, int64_t nf, InferSmem &S, EventCounts &k)
{
    const SpeciesPtrs<T> &P = g.parent, &G = g.out0;
    const unsigned lane = threadIdx.x & 31u;
    const int64_t e = base + lane;
    const int64_t i0 = e < nf ? g.fire_idx[e] : -1;
    const bool valid = i0 >= 0 && i0 < P.cap;  // entries outside the parent are ignored
    const int64_t i = valid ? i0 : 0;
    const T chi = valid ? (T)g.fire_chi[e] : T(0);
    const T px = valid ? P.px[i] : T(0), py = valid ? P.py[i] : T(0), pz = valid ? P.pz[i] : T(1);
    const uint64_t pid = valid ? P.id[i] : 0;

    const U4 w = draw(c.seed, pid, step, kSample);
    const double u = uniform53(w.x, w.y);
    T xi;
    if constexpr (MLP) {
        const MlpIn in = mlp_input(c.mlpv, (double)chi, u);
        const int wib = threadIdx.x >> 5;
        const float y = mlp_forward_warp(S.net, S.h1[wib], S.y[wib], in.x1, in.x2);
        xi = valid ? (T)mlp_output(QED_PROC_QS, y, in) : T(0);
    } else {
        xi = valid ? qs_sample_xi<T>(c.tab, chi, sample_uniform<T>(u)) : T(0);
    }

    const T p2 = px * px + py * py + pz * pz;
    T inv;  // 1/|p|
    if constexpr (sizeof(T) == 8) {
        inv = p2 > T(0) ? rsqrt(p2) : T(0);  // (within 1 ulp; no FP64 division)
    } else {
        const T pm = d_sqrt(p2);
        inv = pm > T(0) ? T(1) / pm : T(0);
    }
    const T gamma = d_sqrt(T(1) + p2);
    const T gg = (gamma - T(1)) * xi;  // photon energy (§2.2)
    const T g1 = gamma - gg;            // lepton energy after emission
    const T q = (g1 - T(1)) * (g1 + T(1));
    const T pn = d_sqrt(q > T(0) ? q : T(0));
    const T nx = px * inv, ny = py * inv, nz = pz * inv;

    // (the FP32 test against the float threshold decides as the FP64 one does,
    // without FP64 instructions)
    const bool keep = valid && (sizeof(T) == 4 ? (float)gg >= c.threshold_f : (double)gg >= c.threshold);
    const long long slot = warp_reserve(G.count, keep);
    const bool room = !keep || slot < G.cap;
    const bool exec = valid && room;
    k.drop += (valid && !room) ? 1 : 0;
    if (keep && room) {
        const U4 cid = draw(c.seed, pid, step, kChildId);
        const uint64_t child = ((uint64_t)cid.y << 32) | cid.x;
        const bool f = c.copy_fields != 0;
        write_particle<T>(G, slot, gg * nx, gg * ny, gg * nz, f ? P.ex[i] : T(0), f ? P.ey[i] : T(0),
                          f ? P.ez[i] : T(0), f ? P.bx[i] : T(0), f ? P.by[i] : T(0), f ? P.bz[i] : T(0), P.w[i],
                          child, tau_draw(c.seed, child, step, kTauInit), f);
        copy_position<T>(G, slot, P, i);
    }
    if (exec) {
        P.px[i] = pn * nx, P.py[i] = pn * ny, P.pz[i] = pn * nz;
        store_tau<T>(P.tau, P.tau_c, i, tau_draw(c.seed, pid, step, kTauReset));
    }
    k.exec += exec ? 1 : 0;
    k.kept += (keep && room) ? 1 : 0;
    k.disc += (exec && !keep) ? 1 : 0;
}

// pair production for entries [base, base + 32) of a firing list of nf entries
template <typename T, bool MLP>
__device__ __forceinline__ void bw_event_chunk(const EventSeg<T> &g, const EventCommon<T> &c, int64_t step,
                                               int64_t base, int64_t nf, InferSmem &S, EventCounts &k)
{
    const SpeciesPtrs<T> &P = g.parent, &E = g.out0, &Q = g.out1;
    const unsigned lane = threadIdx.x & 31u;
    const int64_t e = base + lane;
    const int64_t i0 = e < nf ? g.fire_idx[e] : -1;
    const bool valid = i0 >= 0 && i0 < P.cap;
    const int64_t i = valid ? i0 : 0;
    const T chi = valid ? (T)g.fire_chi[e] : T(0);
    const T px = valid ? P.px[i] : T(0), py = valid ? P.py[i] : T(0), pz = valid ? P.pz[i] : T(1);
    const uint64_t pid = valid ? P.id[i] : 0;

    const U4 w = draw(c.seed, pid, step, kSample);
    const double u = uniform53(w.x, w.y);
    T xm, xp;  // electron and positron fractions of the photon's chi
    if constexpr (MLP) {
        const MlpIn in = mlp_input(c.mlpv, (double)chi, u);
        const int wib = threadIdx.x >> 5;
        const float y = mlp_forward_warp(S.net, S.h1[wib], S.y[wib], in.x1, in.x2);
        const double em = mlp_output(QED_PROC_BW, y, in);
        xm = valid ? (T)em : T(0);
        xp = valid ? (T)(1.0 - em) : T(0);
    } else {
        bool electron = true;
        const T xs = valid ? bw_sample_xi<T>(c.tab, chi, u, electron) : T(0);
        xm = electron ? xs : T(1) - xs;
        xp = electron ? T(1) - xs : xs;
    }

    const T p2 = px * px + py * py + pz * pz;
    const T gg = d_sqrt(p2);  // photon energy (IEEE: it decides whether a pair is made, as in the oracle)
    T inv;
    if constexpr (sizeof(T) == 8)
        inv = p2 > T(0) ? rsqrt(p2) : T(0);  // (within 1 ulp; no FP64 division)
    else
        inv = gg > T(0) ? T(1) / gg : T(0);
    const bool pair = valid && gg > T(2);  // below 2 m_e c^2 no pair
    const T nx = px * inv, ny = py * inv, nz = pz * inv;
    const T km = (gg - T(2)) * xm, kp = (gg - T(2)) * xp;  // kinetic energies (§2.1)
    const T pmm = d_sqrt(km * (km + T(2))), pmp = d_sqrt(kp * (kp + T(2)));

    const long long se = warp_reserve(E.count, pair);
    const long long sq = warp_reserve(Q.count, pair);
    const bool ok_e = se < E.cap, ok_q = sq < Q.cap;
    const bool room = !pair || (ok_e && ok_q);
    const bool exec = valid && room;
    if (pair && !room) {
        ++k.drop;
        if (ok_e) write_dead<T>(E, se);
        if (ok_q) write_dead<T>(Q, sq);
    }
    if (pair && room) {
        const U4 cid = draw(c.seed, pid, step, kChildId);
        const uint64_t ide = ((uint64_t)cid.y << 32) | cid.x;
        const uint64_t idp = ((uint64_t)cid.w << 32) | cid.z;
        const T ex = P.ex[i], ey = P.ey[i], ez = P.ez[i], bx = P.bx[i], by = P.by[i], bz = P.bz[i], wt = P.w[i];
        write_particle<T>(E, se, pmm * nx, pmm * ny, pmm * nz, ex, ey, ez, bx, by, bz, wt, ide,
                          tau_draw(c.seed, ide, step, kTauInit));
        write_particle<T>(Q, sq, pmp * nx, pmp * ny, pmp * nz, ex, ey, ez, bx, by, bz, wt, idp,
                          tau_draw(c.seed, idp, step, kTauInit));
        copy_position<T>(E, se, P, i);
        copy_position<T>(Q, sq, P, i);
        // the photon is removed
        P.w[i] = T(0);
        P.tau[i] = T(INFINITY);
        if (sizeof(T) == 4) P.tau_c[i] = T(0);
    }
    if (valid && !pair) store_tau<T>(P.tau, P.tau_c, i, tau_draw(c.seed, pid, step, kTauReset));
    k.exec += exec ? 1 : 0;
    k.pairs += (pair && room) ? 1 : 0;
    k.nopair += (valid && !pair) ? 1 : 0;
}

__device__ __forceinline__ void flush_counts(long long *stats, const EventCounts &k, bool qs)
{
    if (k.drop) note_error(QED_EW_CAPACITY);
    if (!stats) return;
    if (qs) {
        warp_count(stats + QED_STAT_QS_EVENTS, k.exec);
        warp_count(stats + QED_STAT_PHOTONS_KEPT, k.kept);
        warp_count(stats + QED_STAT_PHOTONS_DISCARDED, k.disc);
    } else {
        warp_count(stats + QED_STAT_BW_EVENTS, k.exec);
        warp_count(stats + QED_STAT_PAIRS, k.pairs);
        warp_count(stats + QED_STAT_BW_NO_PAIR, k.nopair);
    }
    warp_count(stats + QED_STAT_DROPPED_CAPACITY, k.drop);
}

}  // namespace qed
