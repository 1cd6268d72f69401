/*
 * qed.h -- C ABI of libqed, a GB300 (sm_103a) implementation of the per-particle
 * strong-field QED Monte Carlo substep of PICSAR-QED (Fedeli et al., arXiv
 * 2110.00256): optical-depth evolution, quantum-synchrotron (QS) photon emission
 * and nonlinear Breit-Wheeler (BW) pair production.
 *
 * Units (one normalised system): momentum in m_e c; E in the Schwinger field
 * E_s = m_e^2 c^3 / (q_e hbar) (§2); B in E_s / c; time in hbar / (m_e c^2).
 * Then the rates are dN/dt = (2/3) alpha G(chi) / gamma for QS (Eq.
 * (qs_total_cross)) and dN/dt = alpha chi_g T(chi_g) / gamma_g for BW (Eq.
 * (bw_cross_tot)), alpha = 7.2973525693e-3.
 *
 * Conventions for every entry point:
 *  - The return value is a qed_status; QED_OK = 0.  On error nothing has been
 *    enqueued and qed_last_error_message() (thread-local) says why.  No C++
 *    exception crosses this boundary.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  The per-step calls (evolution, events, substeps, pushes,
 *    Schwinger pairs, sampling, training steps) only enqueue work and return
 *    without synchronising; they never allocate device memory and are safe to
 *    capture in a CUDA graph.  Creating tables, batches and networks, and the
 *    launch-shape tuner, allocate and/or synchronise, as stated with each.
 *  - Particle buffers are owned by the caller (device memory, structure of
 *    arrays).  Tables are owned by the library through an opaque handle.
 *  - A pointer documented as "device" must be device memory of the current
 *    device; "host" means ordinary host memory.
 */
#ifndef QED_H
#define QED_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t qed_status;
enum {
    QED_OK = 0,
    QED_ERR_INVALID_ARG = 1, /* a NULL, misaligned or out-of-range argument            */
    QED_ERR_CUDA = 2,        /* a CUDA runtime call failed (message has the CUDA error)  */
    QED_ERR_CAPACITY = 3,    /* reported through QED_STAT_DROPPED_CAPACITY, see below    */
    QED_ERR_NUMERIC = 4,     /* non-finite input seen (also counted in the stats)         */
    QED_ERR_TIMEOUT = 5,     /* a bounded wait gave up                                    */
    QED_ERR_IO = 6,          /* file could not be read/written or has a bad header       */
    QED_ERR_UNSUPPORTED = 7  /* parameter combination not built into this library         */
};

typedef enum { QED_F32 = 0, QED_F64 = 1 } qed_precision;
typedef enum { QED_PROC_QS = 0, QED_PROC_BW = 1 } qed_process;

/* Axis of one process's tables (§3.1, §3.2).  chi grid: n_chi points
 * log-spaced on [chi_min, chi_max], both ends included.  xi grid of the 2-D
 * table: QS, n_xi points log-spaced on [xi_min, 1]; BW, n_xi points linearly
 * spaced on [0, 1/2] (xi_min unused).  2 <= n_chi, n_xi <= QED_MAX_TABLE_N. */
typedef struct {
    double chi_min, chi_max;
    int32_t n_chi, n_xi;
    double xi_min;
} qed_table_axis;

typedef struct {
    qed_table_axis qs, bw;
} qed_table_params;

#define QED_MAX_TABLE_N 1024

typedef struct qed_tables qed_tables; /* opaque, library-owned */

/* One species, structure of arrays, caller-owned device memory.
 * px..bz, tau, weight: element type float (QED_F32) or double (QED_F64),
 * `capacity` elements each.  tau_c: FP32 only, the Kahan compensation of tau
 * (the optical depth is tau - tau_c); ignored (may be NULL) for QED_F64.
 * id: per-particle 64-bit identifier, the counter of every random draw.
 * d_count: device int64, number of live particles (read by every kernel, grown
 * by the event kernels that append to this species).
 * Vector loads are used when every array is 16-byte aligned. */
typedef struct {
    void *px, *py, *pz;
    void *ex, *ey, *ez;
    void *bx, *by, *bz;
    void *tau, *tau_c, *weight;
    uint64_t *id;
    int64_t capacity;
    int64_t *d_count;
    void *x, *y, *z; /* optional positions (element type as px; NULL when not tracked):
                        products inherit their parent's position */
} qed_species;

/* Device list of the particles whose optical depth went negative in the
 * last evolution: index into the species, and the chi it had (FP64). */
typedef struct {
    int64_t *idx;     /* device, `capacity` entries                    */
    double *chi;      /* device, `capacity` entries                    */
    int64_t *d_count; /* device int64, number of entries               */
    int64_t capacity; /* >= the species capacity, or entries are lost  */
} qed_fire_list;

/* Device counters, accumulated (never reset by the library).  int64 each. */
enum {
    QED_STAT_QS_EVENTS = 0,          /* photon emissions executed                         */
    QED_STAT_BW_EVENTS = 1,          /* photon decays executed (pair or below threshold)  */
    QED_STAT_PHOTONS_KEPT = 2,       /* photons appended                                  */
    QED_STAT_PHOTONS_DISCARDED = 3,  /* photons below the keep threshold (§5)             */
    QED_STAT_PAIRS = 4,              /* e-/e+ pairs appended                              */
    QED_STAT_BW_NO_PAIR = 5,         /* decays of photons with gamma_g <= 2 (no pair)     */
    QED_STAT_DROPPED_CAPACITY = 6,   /* events not executed: a destination was full       */
    QED_STAT_NONFINITE = 7,          /* particles with non-finite chi or optical depth    */
    QED_STAT_FIRE_OVERFLOW = 8,      /* firing particles beyond the fire-list capacity    */
    QED_STAT_WAIT_TIMEOUT = 9,       /* CTAs that gave up a bounded wait of the copy
                                        pipeline (never expected; the launch's results
                                        are then incomplete)                             */
    QED_STAT_SCHWINGER_PAIRS = 10,   /* pairs made by qed_schwinger_pairs                  */
    QED_STAT_EVOLVED = 11,           /* particles the batched calls (qed_substep_batched,
                                        qed_push_substep_batched) evolved: each step adds
                                        the live count of every species of every patch,
                                        less the photons that pair production removed and
                                        qed_compact_species has not yet dropped
                                        (QED_STAT_PAIRS - QED_STAT_COMPACTED of the same
                                        array), so the sum over steps is the particle-steps
                                        done                                              */
    QED_STAT_COMPACTED = 12,         /* removed particles dropped by qed_compact_species    */
    QED_STAT_COUNT = 13
};

typedef struct {
    double photon_threshold; /* photons with gamma_g below this are not kept, the emitter
                                still recoils (§5); 0 keeps every photon                     */
    int32_t sampler;         /* 0: 2-D inverse-CDF tables; 1: learned sampler (qed_mlp)       */
    const void *mlp;         /* the qed_mlp* when sampler == 1                                */
    int64_t *d_stats;        /* device int64[QED_STAT_COUNT], or NULL                         */
    void *evolve_begin;      /* optional cudaEvent_t recorded on the stream right before the
                                evolution launch of qed_substep (timing); NULL: none          */
    void *evolve_end;        /* optional cudaEvent_t recorded right after that launch         */
    int64_t *d_step;         /* optional device int64: if set, the step number (a Philox
                                counter word) is read from it instead of the `step`
                                argument; qed_substep and qed_substep_batched add one to it
                                at the end, so that one captured graph replays many steps   */
    int32_t evolve_threads;  /* evolution launch shape: threads per CTA (128, 256 or 512) and */
    int32_t evolve_ctas_per_sm; /* CTAs per SM (1..8); 0 = the library's default / tuned   */
    int32_t evolve_pipeline; /* qed_substep's evolution kernel: QED_EVOLVE_DEFAULT, _DIRECT or
                                _BULK (see below)                                            */
    double qs_chi_cut;       /* leptons with chi below this neither evolve their optical depth
                                nor emit (the cut-off a PIC code applies to photon emission,
                                §5); 0 = off                                                  */
    double bw_chi_cut;       /* the same for photons and pair production; 0 = off           */
    int64_t wait_limit_cycles; /* limit, in SM clock cycles, of the waits between the producer
                                warp and the consumer warps of the bulk-copy evolution (single
                                and batched); 0 = the default of ~1 s.  A wait that runs out
                                ends the CTA's work early (its particles are not evolved),
                                counts QED_STAT_WAIT_TIMEOUT and sets QED_EW_WAIT_TIMEOUT; the
                                producer still waits, with the full limit, for every copy it
                                issued before the CTA exits.  Small values only serve to test
                                that path                                                    */
} qed_substep_opts;

/* How qed_substep's evolution reads the particle arrays.  DIRECT: every thread
 * loads its particles with 16-byte loads into registers.  BULK (FP32, arrays
 * 16-byte aligned; otherwise DIRECT): a producer warp per CTA copies whole
 * tiles of every array into shared-memory stages with the bulk-copy engine,
 * consumer warps evaluate them; evolve_threads 512 (16 consumer warps, 2
 * stages) or evolve_ctas_per_sm 2 (8 warps, 2 stages) pick other shapes than
 * the default (8 consumer warps, 4 stages, 1 CTA per SM).  DIRECT in FP32
 * runs 4 CTAs of 256 threads per SM (64 registers), or 3 (80 registers) with
 * evolve_ctas_per_sm 3.  All give identical results.  DEFAULT (with
 * evolve_threads and evolve_ctas_per_sm 0) is a bulk-copy pipeline with 15
 * consumer warps and 2 stages in FP32 when the arrays are 16-byte aligned, the
 * fastest on GB300, and DIRECT otherwise. */
enum { QED_EVOLVE_DEFAULT = 0, QED_EVOLVE_DIRECT = 1, QED_EVOLVE_BULK = 2 };

/* ------------------------------------------------------------------------- */
/* library                                                                   */
/* ------------------------------------------------------------------------- */
const char *qed_last_error_message(void);
const char *qed_version(void);

/* Device error word.  The per-step calls only enqueue work, so what goes wrong
 * on the device cannot be their return value: their kernels OR these bits into
 * a word that the library keeps on every device, whether or not the caller
 * passed a statistics array (the QED_STAT_* counters give the counts). */
enum {
    QED_EW_WAIT_TIMEOUT = 1u,  /* a bounded wait gave up (results of that launch incomplete) */
    QED_EW_NONFINITE = 2u,     /* non-finite chi or optical depth (the particle never fires) */
    QED_EW_CAPACITY = 4u,      /* an event was not executed: a destination species was full  */
    QED_EW_FIRE_OVERFLOW = 8u  /* firing particles beyond a firing list's capacity            */
};
/* Synchronise `stream`, then read the current device's error word into
 * *word_out (may be NULL) and clear it if `clear` != 0.  Returns QED_ERR_TIMEOUT
 * if QED_EW_WAIT_TIMEOUT is set, else QED_ERR_CAPACITY for QED_EW_CAPACITY or
 * QED_EW_FIRE_OVERFLOW, else QED_ERR_NUMERIC for QED_EW_NONFINITE, else QED_OK
 * (QED_ERR_CUDA if the stream itself failed).  Not for use inside a stream
 * capture (it synchronises).  The word covers every call on the device since it
 * was last cleared, from any stream or thread. */
qed_status qed_device_status(void *stream, uint32_t *word_out, int32_t clear);

/* ------------------------------------------------------------------------- */
/* units (§3.3: one normalised system inside, conversions at the boundary)    */
/* ------------------------------------------------------------------------- */
/* The SI value of one unit of each quantity of a unit system (CODATA 2018).
 * Converting a value v from system a to system b: v * a.x / b.x. */
typedef struct {
    double length;   /* m     */
    double time;     /* s     */
    double momentum; /* kg m/s */
    double energy;   /* J     */
    double e_field;  /* V/m   */
    double b_field;  /* T     */
} qed_unit_scales;

/* The library's own units: length hbar/(m_e c), time hbar/(m_e c^2), momentum
 * m_e c, energy m_e c^2, E in E_s = m_e^2 c^3/(q_e hbar) (§2, the Schwinger
 * field, ~1.32e18 V/m), B in E_s/c. */
qed_status qed_units_library(qed_unit_scales *out);
/* A PIC code normalised to a reference angular frequency omega_r (rad/s):
 * length c/omega_r, time 1/omega_r, momentum m_e c, energy m_e c^2, E in
 * m_e c omega_r/q_e, B in m_e omega_r/q_e.  Also the reference-length form with
 * omega_r = 2 pi c / lambda_r. */
qed_status qed_units_reference_frequency(double omega_r, qed_unit_scales *out);
qed_status qed_units_reference_length(double lambda_r, qed_unit_scales *out);
/* Heaviside-Lorentz natural units (hbar = c = 1) with 1 MeV as the reference
 * energy: length hbar c/MeV, time hbar/MeV, momentum MeV/c, energy MeV, and
 * fields in MeV^2 (q_e = sqrt(4 pi alpha)). */
qed_status qed_units_heaviside_lorentz_mev(qed_unit_scales *out);

/* ------------------------------------------------------------------------- */
/* tables (§3.1, §3.2; generation §3 and §5)                                  */
/* ------------------------------------------------------------------------- */
/* Build the four tables in FP64 on the GPU (ln G, ln P for QS; ln T, P for BW)
 * by quadrature of the modified Bessel functions (Eqs. (t_func_0),
 * (bw_prob_dist), (qs_g_func), (qs_prob_dist)), and keep FP32 copies rounded
 * to nearest (§3.3: tables may be computed in FP64 and kept in FP32).  Synchronises
 * `stream` before returning.  *out receives a new handle. */
qed_status qed_tables_generate(const qed_table_params *params, qed_tables **out, void *stream);

/* Make tables from host arrays (FP64, row-major [n_chi][n_xi]): qs_lnG[qs.n_chi],
 * qs_lnP[qs.n_chi * qs.n_xi], bw_lnT[bw.n_chi], bw_P[bw.n_chi * bw.n_xi].  The
 * arrays are copied; the caller keeps ownership.  Synchronises `stream`. */
qed_status qed_tables_create(const qed_table_params *params, const double *qs_lnG,
                             const double *qs_lnP, const double *bw_lnT, const double *bw_P,
                             qed_tables **out, void *stream);

/* Copy the FP64 tables into host arrays laid out as for qed_tables_create (any
 * pointer may be NULL to skip that table).  Synchronous. */
qed_status qed_tables_copy_to_host(const qed_tables *t, double *qs_lnG, double *qs_lnP,
                                   double *bw_lnT, double *bw_P);

qed_status qed_tables_get_params(const qed_tables *t, qed_table_params *out);

/* Binary file: magic, version, params, the four FP64 arrays, a 64-bit
 * checksum.  Load verifies all of them and returns QED_ERR_IO on mismatch. */
qed_status qed_tables_save(const qed_tables *t, const char *path);
qed_status qed_tables_load(const char *path, qed_tables **out, void *stream);

qed_status qed_tables_destroy(qed_tables *t);

/* ------------------------------------------------------------------------- */
/* optical depth (§3)                                                         */
/* ------------------------------------------------------------------------- */
/* tau = -ln U for particles [0, *d_count), U the 53-bit Philox4x32-10 uniform of
 * (key = seed, counter = (id, step, 2)), computed in FP64; for QED_F32 tau_c
 * receives the rounding residual so that tau - tau_c keeps the FP64 value. */
qed_status qed_init_optical_depth(const qed_species *sp, qed_precision prec, uint64_t seed,
                                  int64_t step, void *stream);

/* Evolve the optical depth of every particle of `sp` (§3, Fig. scheme):
 * chi from its definition in §2 (lepton or photon), rate from the 1-D table (log-log interpolation of
 * §3.1/§3.2; QS clamps outside the table, BW uses the asymptotes of Eq.
 * (t_func)), tau -= rate * dt (FP32: Kahan-compensated with tau_c).  Particles
 * whose optical depth becomes negative are appended to `fire` (index and chi);
 * fire->d_count is reset by this call.  `stats` may be NULL. */
qed_status qed_evolve_optical_depth(const qed_tables *t, qed_process proc, const qed_species *sp,
                                    double dt, qed_precision prec, const qed_fire_list *fire,
                                    int64_t *d_stats, void *stream);

/* ------------------------------------------------------------------------- */
/* events                                                                    */
/* ------------------------------------------------------------------------- */
/* Photon emission for the firing leptons in `fire` (§2.2, §3.2): xi by
 * inverse-CDF sampling of the 2-D table with U from (seed, (id, step, 0)),
 * gamma_g = (gamma - 1) xi along p; the lepton keeps its direction with
 * gamma' = gamma - gamma_g; its optical depth is reset to -ln U(id, step, 1).
 * The photon (id from (id, step, 3), tau from its own id and purpose 2, the
 * parent's weight, E and B) is appended to `photons` if gamma_g >=
 * opts->photon_threshold.  If `photons` is full the event is not executed (the
 * lepton keeps tau < 0 and fires again next step) and
 * QED_STAT_DROPPED_CAPACITY counts it. */
qed_status qed_generate_photons(const qed_tables *t, const qed_species *leptons,
                                const qed_species *photons, const qed_fire_list *fire,
                                uint64_t seed, int64_t step, const qed_substep_opts *opts,
                                qed_precision prec, void *stream);

/* Pair production for the firing photons in `fire` (§2.1, §3.1): r from
 * (seed, (id, step, 0)); r <= 1/2 samples the electron's xi, otherwise the
 * positron's with r -> 1 - r; K_pm = (gamma_g - 2) xi_pm, both along the photon
 * momentum.  The photon is removed (weight 0, tau = +inf).  gamma_g <= 2 makes
 * no pair: the photon stays, tau reset from purpose 1.  Capacity as above (an
 * event needs a slot in both lepton species). */
qed_status qed_generate_pairs(const qed_tables *t, const qed_species *photons,
                              const qed_species *electrons, const qed_species *positrons,
                              const qed_fire_list *fire, uint64_t seed, int64_t step,
                              const qed_substep_opts *opts, qed_precision prec, void *stream);

/* The whole substep on three species in four launches: zero the firing
 * counts; one evolution launch over electrons (QS), positrons (QS) and photons
 * (BW); one event launch for the three firing lists (photon emission of both
 * leptons and pair production side by side: they touch disjoint particles;
 * with the learned sampler, one launch per list); clamp the counts.  fire[0..2]
 * are the firing lists of the three species in that order.  Products are
 * appended after the live particles and are first evolved in the next call.
 * Graph-capturable. */
qed_status qed_substep(const qed_tables *t, const qed_species *electrons,
                       const qed_species *positrons, const qed_species *photons, double dt,
                       uint64_t seed, int64_t step, const qed_substep_opts *opts,
                       qed_precision prec, const qed_fire_list *fire, void *stream);

/* ------------------------------------------------------------------------- */
/* species diagnostics and upkeep                                             */
/* ------------------------------------------------------------------------- */
/* Energy of a species (§2.1, §2.2: photon emission conserves gamma + gamma_g,
 * pair production gamma_+ + gamma_- = gamma_g, so the sum over the three
 * species is invariant under the substep).  Adds sum_i w_i E_i over particles
 * [0, *d_count) to d_out[0] and the number of particles with nonzero weight to
 * d_out[1] (device double[2], accumulated, never reset by the library), with
 * E = gamma = sqrt(1 + p^2) for leptons (photon == 0) and E = |p| for photons
 * (photon != 0), in m_e c^2; removed particles (weight 0) add nothing.  FP64
 * sums at either precision; one launch, stream-ordered, graph-capturable. */
qed_status qed_species_energy(const qed_species *sp, qed_precision prec, int32_t photon, double *d_out,
                              void *stream);

/* Drop the removed particles of `sp` -- weight 0 and optical depth +inf, the
 * mark that pair production leaves on a decayed photon (§3.1) -- so that they
 * are no longer read every step.  With n = *d_count, r of them removed and
 * n' = n - r: the live particles at [n', n) move into the removed slots in
 * [0, n'), every array together (p, E, B, tau, tau_c, weight, id, and x, y, z
 * when present), k-th live particle of the tail into the k-th removed slot of the
 * head; then *d_count = n'.  The order of the particles is not kept (every
 * random draw is keyed by id, so the physics does not depend on it).  d_work:
 * device int64 scratch of at least QED_COMPACT_WORK(sp->capacity) entries,
 * owned by the caller, free again when the call's work on `stream` is done.
 * d_stats (may be NULL): QED_STAT_COMPACTED grows by r.  Four launches, no
 * host synchronisation, graph-capturable. */
#define QED_COMPACT_WORK(cap) (2 * (int64_t)(cap) + ((int64_t)(cap) + 2047) / 2048 + 8)
qed_status qed_compact_species(const qed_species *sp, qed_precision prec, int64_t *d_work, int64_t work_capacity,
                               int64_t *d_stats, void *stream);

/* ------------------------------------------------------------------------- */
/* Schwinger pair production (§2.3)                                          */
/* ------------------------------------------------------------------------- */
/* Cells of the field mesh: n cells, structure of arrays in the precision of the
 * call, fields in E_s and E_s/c; cell positions (for the products) or NULL. */
typedef struct {
    const void *ex, *ey, *ez, *bx, *by, *bz;
    const void *x, *y, *z;
    int64_t n;
} qed_cells;

/* Pairs made from the vacuum in every cell during dt (Eq. (shw); normalised:
 * rate = eps eta coth(pi eta/eps) exp(-pi/eps) / (4 pi^2) per hbar/(m_e c)
 * cubed per hbar/(m_e c^2), eps and eta from the field invariants).  Each cell
 * of volume dv draws a Poisson number of pairs of weight `weight` with mean
 * rate dv dt / weight (Philox counter (cell, step, 4): inversion up to a mean
 * of 100, the normal approximation above).  Pairs start at rest (§2.3) with
 * the cell's fields and position, ids from Philox (cell, step, 5 + 256 j) and
 * optical depths from their ids; they are appended to `electrons` and
 * `positrons` (capacity-checked: a pair without room in both is not made and is
 * counted as dropped).  Rate and mean in FP64 at either precision.  d_stats:
 * QED_STAT_SCHWINGER_PAIRS, QED_STAT_DROPPED_CAPACITY and (FP32 fields,
 * 16-byte aligned: streamed through shared memory with bounded waits)
 * QED_STAT_WAIT_TIMEOUT, or NULL. */
qed_status qed_schwinger_pairs(const qed_cells *cells, double dv, double dt, double weight, uint64_t seed,
                               int64_t step, const qed_species *electrons,
                               const qed_species *positrons, qed_precision prec, int64_t *d_stats,
                               void *stream);

/* ------------------------------------------------------------------------- */
/* many patches per launch                                                    */
/* ------------------------------------------------------------------------- */
/* A patch: the three species of one region of the simulation, each with its
 * firing list.  Patch sizes may differ by orders of magnitude. */
typedef struct {
    qed_species electrons, positrons, photons;
    qed_fire_list fire[3]; /* electrons, positrons, photons */
} qed_patch;

#define QED_MAX_PATCHES 1024
typedef struct qed_batch qed_batch; /* opaque, library-owned */

/* Copy the descriptors of n_patches patches (pointers, capacities; host array,
 * not kept) into library-owned device memory.  The particle buffers stay the
 * caller's.  Synchronises `stream`. */
qed_status qed_batch_create(const qed_patch *patches, int32_t n_patches, qed_precision prec,
                            qed_batch **out, void *stream);
qed_status qed_batch_destroy(qed_batch *b);

/* qed_substep for every patch of `b` (§3, §5), in four launches whatever the
 * number of patches: zero the firing counts (and add the live counts to
 * QED_STAT_EVOLVED); one persistent evolution launch over all 3 x n species
 * segments (tiles of every segment form one index space, so uneven patches
 * share the grid; FP32 with aligned arrays streams them through shared memory
 * by default); one event launch over all firing lists (photon emission of the
 * leptons and pair production of the photons side by side; with the learned
 * sampler, one launch per process); one launch clamping the counts (and
 * advancing opts->d_step).  Stream-ordered, allocates nothing,
 * graph-capturable.  Results per patch are those of qed_substep on that patch. */
qed_status qed_substep_batched(const qed_tables *t, const qed_batch *b, double dt, uint64_t seed,
                               int64_t step, const qed_substep_opts *opts, void *stream);

/* Launch-shape tuner: times the evolution kernel of `b` (dry runs that read
 * everything and store nothing, so the particles are untouched): for an FP32
 * batch with 16-byte-aligned arrays the default bulk-copy kernel (a producer
 * warp streams tiles into shared memory), then direct loads with 128, 256 and
 * 512 threads per CTA and every CTA count per SM the registers allow; keeps the
 * fastest in `b` (used by qed_substep_batched unless opts override it).
 * *threads_out = *ctas_per_sm_out = 0 when the default was the fastest.
 * Outputs may be NULL.  Synchronises `stream`. */
qed_status qed_tune_evolve(const qed_tables *t, qed_batch *b, int32_t *threads_out,
                           int32_t *ctas_per_sm_out, float *ms_out, void *stream);

/* ------------------------------------------------------------------------- */
/* particle push in an analytic plane wave (drives the cascade workload)     */
/* ------------------------------------------------------------------------- */
/* Not from the paper, whose substep runs inside a PIC code: a minimal pusher
 * so that the substep can be exercised over many steps.  Units c = m_e = 1;
 * lengths in hbar/(m_e c).  Phase phi = omega (t - direction x) + phase0;
 * E = e0 (0, cos phi, 0) (linear) or e0 (0, cos phi, sin phi) (circular);
 * B = direction x-hat cross E. */
typedef struct {
    double e0;            /* amplitude, units of E_s (= a0 * omega for a0 the normalised amplitude) */
    double omega;         /* angular frequency, units of m_e c^2 / hbar                            */
    double phase0;
    int32_t polarization; /* 0 linear, 1 circular                                                   */
    int32_t direction;    /* +1 or -1: the wave travels along direction * x                         */
} qed_plane_wave;

/* One step of dt at time t for every particle of `sp` (positions required):
 * the fields at (x, t) are written into the species' E and B arrays; leptons
 * (charge -1 or +1) get a relativistic Boris push (J. P. Boris, 1970), photons
 * (charge 0) fly straight at c; then x += v dt. */
qed_status qed_push_plane_wave(const qed_species *sp, double charge, const qed_plane_wave *wave, double t,
                               double dt, qed_precision prec, void *stream);
/* The same for every species of a batch (electrons -1, positrons +1, photons
 * 0; every species of the batch must have positions) in one launch, at time
 * t0 + step * dt, the step read from d_step when it is not NULL. */
qed_status qed_push_batched(const qed_batch *b, const qed_plane_wave *wave, double t0, double dt,
                            int64_t step, const int64_t *d_step, void *stream);
/* qed_push_batched followed by qed_substep_batched, with the push fused into
 * the evolution: one pass per particle computes the wave's fields at x (time
 * t0 + step * dt, the step read from opts->d_step when set), pushes, and
 * evolves the optical depth on the same registers, so that positions, momenta
 * and optical depths cross HBM once per step.  The particles end bit for bit as
 * with the two separate calls; the species' E and B arrays are written only if
 * store_fields != 0 (otherwise they are left alone, and the photons emitted
 * get no field values: the next step computes every particle's fields before
 * any use).  Graph-capturable. */
qed_status qed_push_substep_batched(const qed_tables *t, const qed_batch *b, const qed_plane_wave *wave,
                                    double t0, double dt, uint64_t seed, int64_t step,
                                    const qed_substep_opts *opts, int32_t store_fields, void *stream);
/* One step of dt for every particle of `sp` (positions required) in the fields
 * already stored in its E and B arrays (uniform static fields, or fields a PIC
 * code gathered at the particles): Boris push for charge -1 or +1, straight
 * flight for charge 0, then x += v dt.  The fields are not changed; products of
 * the substep inherit their parent's, so a uniform field stays set. */
qed_status qed_push_stored_fields(const qed_species *sp, double charge, double dt, qed_precision prec,
                                  void *stream);

/* ------------------------------------------------------------------------- */
/* learned sampler (stands in for the 2-D tables of §3.1, §3.2)              */
/* ------------------------------------------------------------------------- */
/* Two small networks, one per process, each 2 -> 64 -> 64 -> 1 with the tanh
 * form of GELU, bf16 weights and FP32 accumulation; the 64x64 layer runs on the
 * tensor cores.  Input features: x1 = ln chi scaled to [-1, 1] over the
 * tables' chi range (chi clamped into it), x2 = 2 U - 1 (QS) or 2 (2 min(U,
 * 1 - U)) - 1 (BW).  Outputs: QS, y = ln xi - 3 ln U (xi = exp(min(y + 3 ln U,
 * 0))); BW, y = the fraction of the lepton that U selects (U <= 1/2: the
 * electron, as in §3.1), clamped to [0, 1/2].  Trained by the library's own
 * forward/backward kernels with Adam on the mean squared error of y against
 * (chi, U, xi) samples, xi typically from qed_table_sample on fine FP64 tables.
 * qed_substep / qed_generate_* use it when opts->sampler == 1 and opts->mlp
 * points to a qed_mlp.  Parameter vector: QED_MLP_PARAMS floats, W1[64][2],
 * b1[64], W2[64][64], b2[64], W3[64], b3. */
#define QED_MLP_PARAMS 4417
typedef struct qed_mlp qed_mlp; /* opaque, library-owned */

/* Both networks, Glorot-uniform weights drawn from Philox(seed), zero biases;
 * the input scaling takes the chi ranges of `t`.  Synchronises `stream`. */
qed_status qed_mlp_create(const qed_tables *t, uint64_t seed, qed_mlp **out, void *stream);
qed_status qed_mlp_destroy(qed_mlp *m);
/* Both networks to a file: their chi ranges and FP32 master parameters, with
 * an FNV-1a checksum (the Adam moments are not kept).  Synchronous; the file
 * is overwritten; QED_ERR_IO if it cannot be written. */
qed_status qed_mlp_save(const qed_mlp *m, const char *path);
/* A new qed_mlp (owned by the caller, freed with qed_mlp_destroy) from a file
 * that qed_mlp_save wrote: the chi ranges come from the file, Adam starts
 * afresh.  QED_ERR_IO (and *out = NULL) for a missing, short, corrupted
 * (checksum) or foreign file, or one with non-finite parameters.
 * Synchronises `stream`. */
qed_status qed_mlp_load(const char *path, qed_mlp **out, void *stream);
/* FP32 master parameters of one network to / from host memory (set also
 * refreshes the bf16 copy and clears the Adam moments; synchronous). */
qed_status qed_mlp_get_params(const qed_mlp *m, qed_process proc, float *host_params);
qed_status qed_mlp_set_params(qed_mlp *m, qed_process proc, const float *host_params, void *stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the mean squared error
 * of a batch: device arrays chi[n], u[n], xi[n] (FP64; for BW xi is the
 * electron's fraction chi_-/chi_g).  d_loss (device float, may be NULL)
 * receives the batch loss before the step.  Calls on one network must not
 * overlap.  Deterministic: the same network and batches give the same
 * parameters bit for bit (the per-CTA gradient sums are added in a fixed
 * order). */
qed_status qed_mlp_train_step(qed_mlp *m, qed_process proc, const double *d_chi, const double *d_u,
                              const double *d_xi, int64_t n, float lr, float *d_loss, void *stream);
/* Gradient of the batch loss with respect to the parameter vector (device
 * float[QED_MLP_PARAMS]), no update. */
qed_status qed_mlp_gradients(qed_mlp *m, qed_process proc, const double *d_chi, const double *d_u,
                             const double *d_xi, int64_t n, float *d_grad, float *d_loss, void *stream);
/* Batch inference: xi[i] for (chi[i], u[i]) (QS: chi_gamma/chi; BW: the
 * electron's chi_-/chi_g), device FP64 arrays. */
qed_status qed_mlp_sample(const qed_mlp *m, qed_process proc, const double *d_chi, const double *d_u,
                          int64_t n, double *d_xi, void *stream);
/* The same through the 2-D tables (§3.1, §3.2) in the given precision.  Both
 * samplers accept n = 0 (nothing to do); training and gradients need n > 0. */
qed_status qed_table_sample(const qed_tables *t, qed_process proc, qed_precision prec, const double *d_chi,
                            const double *d_u, int64_t n, double *d_xi, void *stream);

/* The exact inverse CDF, without tables (the learned sampler's training
 * targets, and a reference for both samplers): for each of m values chi[i]
 * (device FP64) and each of k draws u[i k + j] (device FP64 in [0, 1]),
 * xi[i k + j] solves P(chi_i, xi) = u to ~1e-13 relative: QS (§3.2, the
 * number spectrum S(chi, xi)/xi of Eq. (qs_diff_cross)) gives chi_gamma/chi;
 * BW (§3.1, Eq. (bw_prob_dist)) the electron's chi_-/chi_g, u <= 1/2 sampling
 * the electron as in the table path.  FP64 quadrature on the GPU: per chi the
 * cumulative integral over a fine grid of 1024 intervals (Gauss-Legendre; the
 * QS grid is uniform in ln(xi / (1 - xi)), the BW grid in ln xi), per draw the
 * bracketing interval, a cubic Hermite first guess and Newton steps on the
 * partial integral.  d_work: device FP64 scratch of at least QED_EXACT_WORK(m)
 * entries.  Stream-ordered; m < 2^31, m k <= 2^40. */
#define QED_EXACT_WORK(m) ((int64_t)(m) * 2051)
qed_status qed_exact_sample(qed_process proc, const double *d_chi, int64_t m, const double *d_u, int64_t k,
                            double *d_xi, double *d_work, int64_t work_capacity, void *stream);

/* ------------------------------------------------------------------------- */
/* measurement                                                                */
/* ------------------------------------------------------------------------- */
/* Not part of the method: the FP64 throughput of this GPU, measured by a kernel
 * of nothing but dependent fused multiply-add chains (8 per thread, 256 threads
 * per CTA, ctas_per_sm CTAs per SM, `iters` FMAs per chain), timed with CUDA
 * events around one launch after a warm-up launch.  *fma_per_s receives FMA
 * instructions per second (each thread's FMA counted once); d_sink: one device
 * double (never written in practice).  Synchronises `stream`. */
qed_status qed_probe_fp64_fma(int64_t iters, int32_t ctas_per_sm, double *d_sink, double *fma_per_s,
                              float *ms_out, void *stream);
/* Not part of the method: the rate of tanh.approx.f32 on this GPU's
 * special-function units, the operation that bounds the learned sampler's GELUs
 * (two layers of 64 per sample).  The same form as qed_probe_fp64_fma: a kernel
 * of nothing but dependent chains x <- tanh(x) / 2 + 1/2 (8 per thread, 256
 * threads per CTA, ctas_per_sm CTAs per SM, `iters` steps per chain), timed
 * with CUDA events around one launch after a warm-up launch; *tanh_per_s
 * receives tanh evaluations per second.  d_sink: one device double (never
 * written in practice).  Synchronises `stream`. */
qed_status qed_probe_tanh(int64_t iters, int32_t ctas_per_sm, double *d_sink, double *tanh_per_s, float *ms_out,
                          void *stream);
/* Not part of the method: the FP64 logarithm and exponential of the rate
 * lookups (Tang's table-driven forms) beside the CUDA library's, for accuracy
 * checks.  d_out: 4 n device doubles, written as [log_tang(x) | exp_tang(x) |
 * log(x) | exp(x)] for the n device doubles d_x.  Stream-ordered; n <= 2^40. */
qed_status qed_probe_fp64_logexp(const double *d_x, int64_t n, double *d_out, void *stream);

/* ------------------------------------------------------------------------- */
/* the substep without caller-provided working memory                        */
/* ------------------------------------------------------------------------- */
/* The paper has no counterpart to this entry point; it exists for callers of
 * this library that cannot allocate device memory: codes whose GPU memory is
 * owned by their own pool allocator, callers that must not trigger the device
 * synchronisation that cudaMalloc / cudaFree imply in the middle of a time step,
 * and runtimes that forbid allocations after start-up.
 *
 * Same arguments and results as qed_substep, without `fire`: the three firing
 * lists live in a fixed array compiled into libqed (QED_NOALLOC_MAX_PARTICLES
 * entries of index + chi, about 16 MiB), which every GPU that loads the
 * library holds until the process exits.  The three species' capacities
 * together may not exceed QED_NOALLOC_MAX_PARTICLES (QED_ERR_INVALID_ARG
 * otherwise).  No allocation happens in this call.
 *
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) and caches it; make that first call before any stream
 * capture.  The cached address belongs to the device's context of that moment:
 * after cudaDeviceReset (or anything else that destroys the context) this entry
 * point is not usable again in the same process.  All calls share the one array (the firing counts are zeroed on the
 * stream at the start of each call, the lists keep the last call's contents):
 * calls that may overlap on the GPU -- different streams, or different host
 * threads -- race and must be serialised by the caller. */
#define QED_NOALLOC_MAX_PARTICLES (1 << 20)
qed_status qed_substep_noalloc(const qed_tables *t, const qed_species *electrons,
                               const qed_species *positrons, const qed_species *photons, double dt,
                               uint64_t seed, int64_t step, const qed_substep_opts *opts,
                               qed_precision prec, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* QED_H */
