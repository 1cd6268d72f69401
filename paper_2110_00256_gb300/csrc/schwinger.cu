// schwinger.cu -- Schwinger pair production per cell (§2.3, Eq. (shw)).  In
// normalised units (c = 1, fields in E_s) the rate per unit volume and time is
// eps eta coth(pi eta / eps) exp(-pi / eps) / (4 pi^2), in units of
// 1/(lambda_C^3 t_C), with eps, eta from the field invariants F = (E^2 - B^2)/2
// and G = E.B.  Each cell draws a Poisson number of pairs of weight w with mean
// rate dV dt / w (inversion for means up to 100, else the normal approximation
// by Box-Muller; one Philox draw, counter (cell, step, 4)); the pairs start at
// rest with the cell's fields (and position), ids from Philox (cell, step,
// 5 + 256 j) and optical depths from their ids.  The rate and the mean are
// evaluated in FP64 at either storage precision, so that the integer counts do
// not depend on it.
#include <cmath>

#include "launch.cuh"
#include "common.cuh"
#include "physics.cuh"
#include "pipeline.cuh"

namespace qed {

constexpr uint32_t kPoisson = 4u, kPairIds = 5u;
constexpr double kPi = 3.141592653589793;

// the rate of Eq. (shw) in FP64 (out of line, like poisson_draw and make_pairs:
// the rare paths stay out of the streaming loop's registers)
__device__ __noinline__ double schwinger_rate(double ex, double ey, double ez, double bx, double by, double bz)
{
    const double F = 0.5 * ((ex * ex + ey * ey + ez * ez) - (bx * bx + by * by + bz * bz));
    const double G = ex * bx + ey * by + ez * bz;
    const double r = sqrt(F * F + G * G);
    const double eps = sqrt(r + F);
    const double eta = sqrt(r - F > 0.0 ? r - F : 0.0);
    if (!(eps > 0.0)) return 0.0;
    const double x = kPi * eta / eps;  // eta coth(pi eta / eps) = (eps / pi) x coth x
    const double xcothx = x < 1e-8 ? 1.0 : x / tanh(x);
    return eps * (eps / kPi) * xcothx * exp(-kPi / eps) / (4.0 * kPi * kPi);
}

__device__ __noinline__ long long poisson_draw(double lambda, uint64_t seed, uint64_t cell, int64_t step)
{
    if (!(lambda > 0.0)) return 0;
    const U4 w = draw(seed, cell, step, kPoisson);
    const double u = uniform53(w.x, w.y);
    if (lambda <= 100.0) {
        double p = exp(-lambda), cdf = p;
        long long k = 0;
        while (u > cdf && k < 1000) {
            ++k;
            p *= lambda / (double)k;
            cdf += p;
        }
        return k;
    }
    const double z = sqrt(-2.0 * log(u)) * cos(2.0 * kPi * uniform53(w.z, w.w));
    const double k = floor(lambda + sqrt(lambda) * z + 0.5);
    return k > 0.0 ? (long long)k : 0;
}

template <typename T>
struct CellsView {
    const T *ex, *ey, *ez, *bx, *by, *bz, *x, *y, *z;
    int64_t n;
};

template <typename T>
struct PairDest {
    T *px, *py, *pz, *ex, *ey, *ez, *bx, *by, *bz, *tau, *tau_c, *w, *x, *y, *z;
    uint64_t *id;
    unsigned long long *count;
    int64_t cap;
};

template <typename T>
PairDest<T> pair_dest(const qed_species *s)
{
    return PairDest<T>{(T *)s->px, (T *)s->py, (T *)s->pz, (T *)s->ex, (T *)s->ey, (T *)s->ez,
                       (T *)s->bx, (T *)s->by, (T *)s->bz, (T *)s->tau, (T *)s->tau_c, (T *)s->weight,
                       (T *)s->x, (T *)s->y, (T *)s->z, s->id, (unsigned long long *)s->d_count,
                       s->capacity};
}

template <typename T>
__device__ __forceinline__ void put(const PairDest<T> &d, int64_t k, const CellsView<T> &c, int64_t cell, T weight,
                                    uint64_t id, double tau)
{
    d.px[k] = T(0), d.py[k] = T(0), d.pz[k] = T(0);
    d.ex[k] = c.ex[cell], d.ey[k] = c.ey[cell], d.ez[k] = c.ez[cell];
    d.bx[k] = c.bx[cell], d.by[k] = c.by[cell], d.bz[k] = c.bz[cell];
    d.w[k] = weight;
    d.id[k] = id;
    store_tau<T>(d.tau, d.tau_c, k, tau);
    if (d.x && c.x) d.x[k] = c.x[cell], d.y[k] = c.y[cell], d.z[k] = c.z[cell];
}

// a slot reserved for a pair whose other half found no room
template <typename T>
__device__ __forceinline__ void put_dead(const PairDest<T> &d, int64_t k)
{
    d.px[k] = T(0), d.py[k] = T(0), d.pz[k] = T(0);
    d.ex[k] = T(0), d.ey[k] = T(0), d.ez[k] = T(0), d.bx[k] = T(0), d.by[k] = T(0), d.bz[k] = T(0);
    d.w[k] = T(0);
    d.id[k] = ~0ull;
    store_tau<T>(d.tau, d.tau_c, k, (double)INFINITY);
    if (d.x) d.x[k] = T(0), d.y[k] = T(0), d.z[k] = T(0);
}

// add per-lane 64-bit counts to a device counter, one atomic per warp
__device__ __forceinline__ void warp_count64(long long *ctr, long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31u) == 0 && v) atomicAdd((unsigned long long *)ctr, (unsigned long long)v);
}

// warp-aggregated reservation of v slots per lane: one atomic per warp
__device__ __forceinline__ long long warp_reserve_n(unsigned long long *counter, long long v)
{
    const unsigned lane = threadIdx.x & 31u;
    long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o) incl += t;
    }
    const long long total = __shfl_sync(0xffffffffu, incl, 31);
    unsigned long long base = 0;
    if (lane == 31 && total > 0) base = atomicAdd(counter, (unsigned long long)total);
    base = __shfl_sync(0xffffffffu, base, 31);
    return (long long)base + incl - v;
}

// VEC consecutive cells per thread (16-byte loads when the arrays allow); a
// warp whose cells make no pair skips the reservation
template <typename T, int VEC>
__device__ __forceinline__ void load_cells(const T *a, int64_t i0, int64_t n, bool vec, T (&v)[VEC])
{
    if constexpr (VEC == 4) {
        if (vec && i0 + 4 <= n) {
            const float4 q = __ldcs(reinterpret_cast<const float4 *>(a + i0));
            v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
            return;
        }
    } else if constexpr (VEC == 2) {
        if (vec && i0 + 2 <= n) {
            const double2 q = __ldcs(reinterpret_cast<const double2 *>(a + i0));
            v[0] = q.x, v[1] = q.y;
            return;
        }
    }
#pragma unroll
    for (int j = 0; j < VEC; ++j) v[j] = i0 + j < n ? a[i0 + j] : T(0);
}

// The Poisson number of pairs of one cell.
template <typename T>
__device__ __forceinline__ long long cell_pairs(T ex, T ey, T ez, T bx, T by, T bz, int64_t cell, double dv, double dt,
                                                double weight, uint64_t seed, int64_t step, float ln_scale)
{
    // Cells whose mean is below 2^-55 draw no pair whatever U (the largest
    // uniform is 1 - 2^-54, below exp(-mean)).  A FP32 upper bound of the mean
    // skips them: eps_up >= eps (eps^2 = sqrt(F^2 + G^2) + F plus a bound on its
    // rounding, 1e-6 (E^2 + B^2)), eta coth(pi eta/eps) <= eta + eps/pi with
    // eta <= sqrt(E^2 + B^2), and a margin of e^7 against FP32 rounding
    const float fex = (float)ex, fey = (float)ey, fez = (float)ez;
    const float fbx = (float)bx, fby = (float)by, fbz = (float)bz;
    const float e2 = fex * fex + fey * fey + fez * fez, b2 = fbx * fbx + fby * fby + fbz * fbz;
    const float g = fex * fbx + fey * fby + fez * fbz, f = 0.5f * (e2 - b2);
    // First a cheaper, looser bound from reciprocal square roots (each
    // within 2 ulp, widened by 1e-6) and ln x <= x - 1, which settles
    // the cells of PIC-strength fields; q >= eps_up^2 below.  q <= 0 with
    // finite fields means eps = 0: no pair.
    const float s2 = e2 + b2, r2 = f * f + g * g;
    const float q = (r2 > 0.0f ? r2 * rsqrtf(r2) * 1.000001f : 0.0f) + f + 1.0e-6f * s2;
    if (!(q > 0.0f) && q == q && s2 == s2) return 0;
    {
        const float rq = rsqrtf(q);
        const float eps_hi = q * rq * 1.000001f, pi_over_lo = 3.1415925f * rq * 0.999999f;
        const float s_hi = (s2 > 0.0f ? s2 * rsqrtf(s2) : 0.0f) * 1.000001f;
        if (eps_hi * (s_hi + eps_hi) - 1.0f - pi_over_lo + ln_scale < -45.0f) return 0;
    }
    const float eps_up = sqrtf(sqrtf(f * f + g * g) + f + 1.0e-6f * (e2 + b2));
    const float ln_up = logf(eps_up * (sqrtf(e2 + b2) + eps_up)) - 3.14159274f / eps_up + ln_scale;
    if (ln_up < -45.0f) return 0;  // -55 ln 2 = -38.1
    const double rate = schwinger_rate((double)ex, (double)ey, (double)ez, (double)bx, (double)by, (double)bz);
    return poisson_draw(rate * dv * dt / weight, seed, (uint64_t)cell, step);
}

// the pairs of a warp's cells (rare; every lane of the warp calls it): the
// counts again, slots reserved with one atomic per warp and species, the pairs
// written.  The streaming loops keep no per-cell array alive for it.
template <typename T, int VEC>
__device__ __noinline__ void make_pairs(int64_t c0, const CellsView<T> &c, double dv, double dt, double weight,
                                        uint64_t seed, int64_t step, float ln_scale, const PairDest<T> &e,
                                        const PairDest<T> &p, long long &made, long long &dropped)
{
    // the counts again, from the cells in global memory (the same draws: counter-based)
    long long k[VEC], tot = 0;
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
        k[j] = c0 + j < c.n ? cell_pairs<T>(c.ex[c0 + j], c.ey[c0 + j], c.ez[c0 + j], c.bx[c0 + j], c.by[c0 + j],
                                            c.bz[c0 + j], c0 + j, dv, dt, weight, seed, step, ln_scale)
                            : 0;
        tot += k[j];
    }
    const long long se = warp_reserve_n(e.count, tot);
    const long long sp = warp_reserve_n(p.count, tot);
    long long off = 0;
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
        const int64_t cell = c0 + j;
        // slots [se + off, se + off + k) and [sp + off, ...); only those below the
        // capacities exist, so the loop ends with the last of them whatever k is
        const long long be = se + off, bp = sp + off;
        const long long room_e = e.cap - be > 0 ? e.cap - be : 0, room_p = p.cap - bp > 0 ? p.cap - bp : 0;
        const long long both = room_e < room_p ? room_e : room_p, any = room_e > room_p ? room_e : room_p;
        const long long n_made = k[j] < both ? k[j] : both, n_touch = k[j] < any ? k[j] : any;
        for (long long i = 0; i < n_touch; ++i) {
            if (i < n_made) {
                const U4 w = draw(seed, (uint64_t)cell, step, kPairIds + 256u * (uint32_t)i);
                const uint64_t ide = ((uint64_t)w.y << 32) | w.x, idp = ((uint64_t)w.w << 32) | w.z;
                put<T>(e, be + i, c, cell, (T)weight, ide, tau_draw(seed, ide, step, kTauInit));
                put<T>(p, bp + i, c, cell, (T)weight, idp, tau_draw(seed, idp, step, kTauInit));
            } else {  // room in one species only: a placeholder there
                if (i < room_e) put_dead<T>(e, be + i);
                if (i < room_p) put_dead<T>(p, bp + i);
            }
        }
        made += n_made;
        dropped += k[j] - n_made;
        off += k[j];
    }
}

// ln_scale = ln(dv dt / (weight 4 pi^2)), in FP32 (+inf when it overflows).
// 3 CTAs of 256 per SM (80 registers): faster than 4 (64 registers, spills).
template <typename T, int VEC>
__global__ void __launch_bounds__(256, 3) schwinger_kernel(CellsView<T> c, double dv, double dt, double weight,
                                                            uint64_t seed, int64_t step, PairDest<T> e,
                                                            PairDest<T> p, long long *stats, int vec, float ln_scale)
{
    const unsigned lane = threadIdx.x & 31u;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * VEC;
    long long made = 0, dropped = 0;
    // whole warps iterate together (the reservation is warp-collective): the loop
    // runs while the warp's first cell is in range
    for (int64_t c0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) * VEC; c0 - (int64_t)lane * VEC < c.n;
         c0 += stride) {
        T ex[VEC], ey[VEC], ez[VEC], bx[VEC], by[VEC], bz[VEC];
        load_cells<T, VEC>(c.ex, c0, c.n, vec, ex);
        load_cells<T, VEC>(c.ey, c0, c.n, vec, ey);
        load_cells<T, VEC>(c.ez, c0, c.n, vec, ez);
        load_cells<T, VEC>(c.bx, c0, c.n, vec, bx);
        load_cells<T, VEC>(c.by, c0, c.n, vec, by);
        load_cells<T, VEC>(c.bz, c0, c.n, vec, bz);
        long long tot = 0;
#pragma unroll
        for (int j = 0; j < VEC; ++j)
            if (c0 + j < c.n)
                tot += cell_pairs<T>(ex[j], ey[j], ez[j], bx[j], by[j], bz[j], c0 + j, dv, dt, weight, seed, step,
                                     ln_scale);
        if (__any_sync(0xffffffffu, tot > 0))
            make_pairs<T, VEC>(c0, c, dv, dt, weight, seed, step, ln_scale, e, p, made, dropped);
    }
    if (dropped) note_error(QED_EW_CAPACITY);
    if (stats) {
        warp_count64(stats + QED_STAT_SCHWINGER_PAIRS, made);
        warp_count64(stats + QED_STAT_DROPPED_CAPACITY, dropped);
    }
}

// FP32 cells with 16-byte-aligned field arrays: the bulk-copy form.  The last
// warp of the CTA copies whole tiles (TP = CW x 32 x 4 cells) of the six field
// components into S shared-memory stages with cp.async.bulk (completion counted
// on the stage's mbarrier); the CW consumer warps take four cells each from the
// stage, release it, and settle the cells.  The ragged last tile is read from
// global memory.  Every wait is bounded; a warp that gives up raises s_abort,
// and QED_STAT_WAIT_TIMEOUT counts the CTA.
constexpr int kCellArrays = 6;

__device__ __forceinline__ bool cell_wait(uint64_t *bar, uint32_t parity, volatile int *abort)
{
    if (mbar_test(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_test(bar, parity)) {
        if (*abort || clock64() - t0 > kWaitCycles) return false;
    }
    return true;
}

__device__ __forceinline__ void cell_give_up(int *abort, long long *stats)
{
    if (atomicExch(abort, 1) == 0) {
        note_error(QED_EW_WAIT_TIMEOUT);
        if (stats) atomicAdd((unsigned long long *)(stats + QED_STAT_WAIT_TIMEOUT), 1ull);
    }
}

template <int CW, int S>
__global__ void __launch_bounds__((CW + 1) * 32, 1)
    schwinger_bulk_kernel(CellsView<float> c, double dv, double dt, double weight, uint64_t seed, int64_t step,
                          PairDest<float> e, PairDest<float> p, long long *stats, float ln_scale)
{
    constexpr int TP = CW * 32 * 4;
    extern __shared__ __align__(128) float s_stage[];  // [S][kCellArrays][TP]
    __shared__ __align__(8) uint64_t s_full[S];
    __shared__ __align__(8) uint64_t s_empty[S];
    __shared__ int s_abort;
    if (threadIdx.x == 0) {
        s_abort = 0;
        for (int k = 0; k < S; ++k) {
            mbar_init(&s_full[k], 1);
            mbar_init(&s_empty[k], CW);
        }
        mbar_fence_init();
    }
    __syncthreads();
    const long long total = (c.n + TP - 1) / TP;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    volatile int *abort = &s_abort;
    const float *arr[kCellArrays] = {c.ex, c.ey, c.ez, c.bx, c.by, c.bz};

    if (warp == CW) {  // producer
        const uint64_t pol = l2_evict_first();
        int k = 0;
        for (long long t = blockIdx.x; t < total; t += gridDim.x, ++k) {
            const int st = k % S;
            const uint32_t ph = (uint32_t)(k / S) & 1u;
            const int64_t base = t * (int64_t)TP;
            if (!__all_sync(0xffffffffu, cell_wait(&s_empty[st], ph ^ 1u, abort))) {
                if (lane == 0) cell_give_up(&s_abort, stats);
                break;
            }
            if (base + TP <= c.n) {
                if (lane == 0) mbar_arrive_expect_tx(&s_full[st], kCellArrays * TP * (uint32_t)sizeof(float));
                __syncwarp();
                if (lane < kCellArrays)
                    bulk_g2s(s_stage + ((size_t)st * kCellArrays + lane) * TP, arr[lane] + base,
                             TP * (uint32_t)sizeof(float), &s_full[st], pol);
            } else if (lane == 0) {
                mbar_arrive(&s_full[st]);
            }
        }
        // leave only once the copies of the last S tiles have landed
        for (int j = 1; j <= S && j <= k; ++j) {
            const int kk = k - j;
            if (!mbar_wait(&s_full[kk % S], (uint32_t)(kk / S) & 1u) && lane == 0) cell_give_up(&s_abort, stats);
        }
        return;
    }

    long long made = 0, dropped = 0;
    int k = 0;
    for (long long t = blockIdx.x; t < total; t += gridDim.x, ++k) {
        const int st = k % S;
        const uint32_t ph = (uint32_t)(k / S) & 1u;
        const int64_t base = t * (int64_t)TP;
        const int64_t c0 = base + 4 * (int64_t)threadIdx.x;
        if (!__all_sync(0xffffffffu, cell_wait(&s_full[st], ph, abort))) {
            if (lane == 0) cell_give_up(&s_abort, stats);
            break;
        }
        float f[kCellArrays][4];
        if (base + TP <= c.n) {
            const float4 *v = reinterpret_cast<const float4 *>(s_stage + (size_t)st * kCellArrays * TP) + threadIdx.x;
#pragma unroll
            for (int a = 0; a < kCellArrays; ++a) {
                const float4 w = v[a * (TP / 4)];
                f[a][0] = w.x, f[a][1] = w.y, f[a][2] = w.z, f[a][3] = w.w;
            }
        } else {
#pragma unroll
            for (int a = 0; a < kCellArrays; ++a) load_cells<float, 4>(arr[a], c0, c.n, true, f[a]);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&s_empty[st]);
        long long tot = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (c0 + j < c.n)
                tot += cell_pairs<float>(f[0][j], f[1][j], f[2][j], f[3][j], f[4][j], f[5][j], c0 + j, dv, dt, weight,
                                         seed, step, ln_scale);
        if (__any_sync(0xffffffffu, tot > 0))
            make_pairs<float, 4>(c0, c, dv, dt, weight, seed, step, ln_scale, e, p, made, dropped);
    }
    if (dropped) note_error(QED_EW_CAPACITY);
    if (stats) {
        warp_count64(stats + QED_STAT_SCHWINGER_PAIRS, made);
        warp_count64(stats + QED_STAT_DROPPED_CAPACITY, dropped);
    }
}

// the species' counts never pass their capacity
__global__ void clamp_pair_counts(unsigned long long *a, int64_t ca, unsigned long long *b, int64_t cb)
{
    if (threadIdx.x == 0) {
        if (*a > (unsigned long long)ca) *a = ca;
        if (*b > (unsigned long long)cb) *b = cb;
    }
}

template <typename T>
static qed_status launch(const qed_cells *cells, double dv, double dt, double weight, uint64_t seed, int64_t step,
                         const qed_species *el, const qed_species *po, int64_t *d_stats, cudaStream_t st)
{
    const CellsView<T> c{(const T *)cells->ex, (const T *)cells->ey, (const T *)cells->ez, (const T *)cells->bx,
                         (const T *)cells->by, (const T *)cells->bz, (const T *)cells->x, (const T *)cells->y,
                         (const T *)cells->z, cells->n};
    bool vec = true;
    for (const void *a : {cells->ex, cells->ey, cells->ez, cells->bx, cells->by, cells->bz})
        vec = vec && ((uintptr_t)a & 15u) == 0;
    const double ln_scale = std::log(dv * dt / (weight * 4.0 * kPi * kPi));
    const float ln_s = ln_scale < 1e30 ? (float)ln_scale : INFINITY;
    if constexpr (sizeof(T) == 4) {
        if (vec) {
            // 15 consumer warps + the producer (16 warps per SM), 4 stages of 1920 cells
            constexpr int CW = 15, S = 4;
            constexpr int dyn = S * kCellArrays * CW * 32 * 4 * (int)sizeof(float);
            static bool attr = false;
            if (!attr) {
                QED_CUDA_TRY(cudaFuncSetAttribute(schwinger_bulk_kernel<CW, S>,
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
                attr = true;
            }
            const int64_t tiles = (cells->n + CW * 128 - 1) / (CW * 128);
            const int g = (int)(tiles < sm_count() ? tiles : sm_count());
            schwinger_bulk_kernel<CW, S><<<g, (CW + 1) * 32, dyn, st>>>(c, dv, dt, weight, seed, step,
                                                                        pair_dest<T>(el), pair_dest<T>(po),
                                                                        (long long *)d_stats, ln_s);
            QED_LAUNCH_CHECK();
            clamp_pair_counts<<<1, 32, 0, st>>>((unsigned long long *)el->d_count, el->capacity,
                                                (unsigned long long *)po->d_count, po->capacity);
            QED_LAUNCH_CHECK();
            return QED_OK;
        }
    }
    constexpr int V = sizeof(T) == 4 ? 4 : 2;
    const int g = resident_grid<schwinger_kernel<T, V>>(256, 0, (cells->n + V - 1) / V);
    schwinger_kernel<T, V><<<g, 256, 0, st>>>(c, dv, dt, weight, seed, step, pair_dest<T>(el), pair_dest<T>(po),
                                              (long long *)d_stats, vec ? 1 : 0, ln_s);
    QED_LAUNCH_CHECK();
    clamp_pair_counts<<<1, 32, 0, st>>>((unsigned long long *)el->d_count, el->capacity,
                                        (unsigned long long *)po->d_count, po->capacity);
    QED_LAUNCH_CHECK();
    return QED_OK;
}

}  // namespace qed

using namespace qed;

extern "C" qed_status qed_schwinger_pairs(const qed_cells *cells, double dv, double dt, double weight, uint64_t seed,
                                          int64_t step, const qed_species *electrons, const qed_species *positrons,
                                          qed_precision prec, int64_t *d_stats, void *stream)
{
    clear_error();
    qed_status s;
    if (!cells) QED_FAIL(QED_ERR_INVALID_ARG, "cells is NULL");
    if (cells->n < 0) QED_FAIL(QED_ERR_INVALID_ARG, "negative number of cells");
    if (cells->n > 0 && (!cells->ex || !cells->ey || !cells->ez || !cells->bx || !cells->by || !cells->bz))
        QED_FAIL(QED_ERR_INVALID_ARG, "a cell field array is NULL");
    if ((s = check_species(electrons, "electrons", prec))) return s;
    if ((s = check_species(positrons, "positrons", prec))) return s;
    if ((electrons->x || positrons->x) && cells->n > 0 && !cells->x)
        QED_FAIL(QED_ERR_INVALID_ARG, "the species have positions: the cells need theirs");
    if (!(dv > 0.0) || !(dt >= 0.0) || !(weight > 0.0) || !std::isfinite(dv) || !std::isfinite(dt) ||
        !std::isfinite(weight))
        QED_FAIL(QED_ERR_INVALID_ARG, "dv and weight must be > 0, dt >= 0");
    if (cells->n == 0) return QED_OK;
    cudaStream_t st = as_stream(stream);
    return prec == QED_F32 ? launch<float>(cells, dv, dt, weight, seed, step, electrons, positrons, d_stats, st)
                           : launch<double>(cells, dv, dt, weight, seed, step, electrons, positrons, d_stats, st);
}
