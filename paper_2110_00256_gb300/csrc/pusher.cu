// pusher.cu -- a minimal particle push, in an analytic plane wave or in the
// fields stored with the particles, to drive the QED substep in a cascade (the
// paper's substep runs inside a PIC code; this is not from the paper).
// Units: c = m_e = 1, momentum in m_e c, fields in E_s and E_s / c, time in
// hbar/(m_e c^2), lengths in hbar/(m_e c); dp/dt = q (E + v x B).  Positions
// at t_n, momenta at t_{n+1/2}: fields at (x_n, t_n) are written into the
// species' field arrays (where the substep reads them), the momentum is
// advanced with the relativistic Boris rotation (J. P. Boris, 1970) and the
// position with the new velocity; photons fly straight at c.
#include <cmath>
#include <cstring>
#include <vector>

#include "launch.cuh"
#include "pusher.cuh"

namespace qed {

// momentum (Boris) and position update of particle i with the fields (ex .. bz)
template <typename T>
__device__ __forceinline__ void advance(const PushSeg<T> &g, int64_t i, T x, T ex, T ey, T ez, T bx, T by, T bz,
                                        T dt)
{
    T px = g.px[i], py = g.py[i], pz = g.pz[i];
    T vx, vy, vz;
    boris_move<T>(g.q, dt, ex, ey, ez, bx, by, bz, px, py, pz, vx, vy, vz);
    if (g.q != T(0)) g.px[i] = px, g.py[i] = py, g.pz[i] = pz;
    g.x[i] = x + vx * dt;
    g.y[i] = g.y[i] + vy * dt;
    g.z[i] = g.z[i] + vz * dt;
}

// plane wave: fields at (x_n, t_n) are written into the species, then the step
template <typename T>
__device__ __forceinline__ void push_one(const PushSeg<T> &g, int64_t i, const WaveT<T> &w, T dt)
{
    const T x = g.x[i];
    T ex, ey, ez, bx, by, bz;
    wave_fields<T>(w, x, ex, ey, ez, bx, by, bz);
    g.ex[i] = ex, g.ey[i] = ey, g.ez[i] = ez, g.bx[i] = bx, g.by[i] = by, g.bz[i] = bz;
    advance<T>(g, i, x, ex, ey, ez, bx, by, bz, dt);
}

template <typename T>
__global__ void __launch_bounds__(256) push_kernel(const PushSeg<T> *__restrict__ segs, int n_seg, WaveParams w,
                                                    double t0, double dt, const int64_t *d_step, int64_t step)
{
    extern __shared__ long long s_dyn[];  // [n_seg] inclusive prefix of particle counts
    __shared__ long long s_warp[8];
    const int per = (n_seg + blockDim.x - 1) / blockDim.x;
    const int s0 = threadIdx.x * per, s1 = min(n_seg, s0 + per);
    long long local = 0;
    for (int s = s0; s < s1; ++s) {
        long long n = *segs[s].count;
        n = n < 0 ? 0 : (n > segs[s].cap ? segs[s].cap : n);
        local += n;
        s_dyn[s] = n;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long incl = local;
    for (int o = 1; o < 32; o <<= 1) {
        const long long v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    long long acc = incl - local;
    for (int w2 = 0; w2 < warp; ++w2) acc += s_warp[w2];
    for (int s = s0; s < s1; ++s) {
        acc += s_dyn[s];
        s_dyn[s] = acc;
    }
    __syncthreads();
    const long long total = s_dyn[n_seg - 1];
    const WaveT<T> wt = wave_at<T>(w, t0 + (double)(d_step ? *d_step : step) * dt);
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
         k += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = n_seg - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (s_dyn[mid] > k)
                hi = mid;
            else
                lo = mid + 1;
        }
        push_one<T>(segs[lo], k - (lo ? s_dyn[lo - 1] : 0), wt, (T)dt);
    }
}

template <typename T>
PushSeg<T> push_seg(const qed_species *s, double q)
{
    PushSeg<T> g;
    g.x = (T *)s->x, g.y = (T *)s->y, g.z = (T *)s->z;
    g.px = (T *)s->px, g.py = (T *)s->py, g.pz = (T *)s->pz;
    g.ex = (T *)s->ex, g.ey = (T *)s->ey, g.ez = (T *)s->ez;
    g.bx = (T *)s->bx, g.by = (T *)s->by, g.bz = (T *)s->bz;
    g.count = s->d_count;
    g.cap = s->capacity;
    g.q = (T)q;
    return g;
}

template PushSeg<float> push_seg<float>(const qed_species *, double);
template PushSeg<double> push_seg<double>(const qed_species *, double);

// one species, its descriptor as a kernel parameter
template <typename T>
__global__ void __launch_bounds__(256) push_single_kernel(const __grid_constant__ PushSeg<T> g, WaveParams w,
                                                          double t, double dt)
{
    const WaveT<T> wt = wave_at<T>(w, t);
    int64_t n = *g.count;
    n = n < 0 ? 0 : (n > g.cap ? g.cap : n);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        push_one<T>(g, i, wt, (T)dt);
}

// fields already stored in the species (uniform fields, or gathered by the caller)
template <typename T>
__global__ void __launch_bounds__(256) push_stored_kernel(const __grid_constant__ PushSeg<T> g, double dt)
{
    int64_t n = *g.count;
    n = n < 0 ? 0 : (n > g.cap ? g.cap : n);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        advance<T>(g, i, g.x[i], g.ex[i], g.ey[i], g.ez[i], g.bx[i], g.by[i], g.bz[i], (T)dt);
}

template <typename T>
qed_status launch_push(const void *d_segs, int n_seg, const WaveParams &w, double t0, double dt,
                       const int64_t *d_step, int64_t step, int64_t capacity, cudaStream_t st)
{
    if (n_seg <= 0) return QED_OK;
    const size_t dyn = (size_t)n_seg * sizeof(long long);
    static bool attr = false;
    if (!attr) {
        QED_CUDA_TRY(cudaFuncSetAttribute(push_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          3 * QED_MAX_PATCHES * (int)sizeof(long long)));
        attr = true;
    }
    push_kernel<T><<<resident_grid<push_kernel<T>>(256, 3 * QED_MAX_PATCHES * sizeof(long long), capacity), 256, dyn,
                     st>>>((const PushSeg<T> *)d_segs, n_seg, w, t0, dt, d_step, step);
    QED_LAUNCH_CHECK();
    return QED_OK;
}

template qed_status launch_push<float>(const void *, int, const WaveParams &, double, double, const int64_t *,
                                       int64_t, int64_t, cudaStream_t);
template qed_status launch_push<double>(const void *, int, const WaveParams &, double, double, const int64_t *,
                                        int64_t, int64_t, cudaStream_t);

qed_status check_wave(const qed_plane_wave *w)
{
    if (!w) QED_FAIL(QED_ERR_INVALID_ARG, "wave is NULL");
    if (!std::isfinite(w->e0) || !(w->omega > 0.0)) QED_FAIL(QED_ERR_INVALID_ARG, "bad wave amplitude/frequency");
    if (w->direction != 1 && w->direction != -1) QED_FAIL(QED_ERR_INVALID_ARG, "wave direction must be +1 or -1");
    return QED_OK;
}

WaveParams wave_params(const qed_plane_wave *w)
{
    const double pi = 3.141592653589793;
    return WaveParams{w->e0, w->omega / pi, w->phase0 / pi, w->polarization == 1 ? 1 : 0, w->direction};
}

}  // namespace qed

using namespace qed;

extern "C" qed_status qed_push_plane_wave(const qed_species *sp, double charge, const qed_plane_wave *wave, double t,
                                          double dt, qed_precision prec, void *stream)
{
    clear_error();
    qed_status s;
    if ((s = check_species(sp, "species", prec))) return s;
    if (!sp->x || !sp->y || !sp->z) QED_FAIL(QED_ERR_INVALID_ARG, "the push needs the species' positions");
    if ((s = check_wave(wave))) return s;
    if (!std::isfinite(dt) || dt < 0) QED_FAIL(QED_ERR_INVALID_ARG, "dt must be finite and >= 0");
    cudaStream_t st = as_stream(stream);
    if (prec == QED_F32)
        push_single_kernel<float><<<resident_grid<push_single_kernel<float>>(256, 0, sp->capacity), 256, 0, st>>>(
            push_seg<float>(sp, charge), wave_params(wave), t, dt);
    else
        push_single_kernel<double><<<resident_grid<push_single_kernel<double>>(256, 0, sp->capacity), 256, 0, st>>>(
            push_seg<double>(sp, charge), wave_params(wave), t, dt);
    QED_LAUNCH_CHECK();
    return QED_OK;
}

extern "C" qed_status qed_push_stored_fields(const qed_species *sp, double charge, double dt, qed_precision prec,
                                             void *stream)
{
    clear_error();
    qed_status s;
    if ((s = check_species(sp, "species", prec))) return s;
    if (!sp->x || !sp->y || !sp->z) QED_FAIL(QED_ERR_INVALID_ARG, "the push needs the species' positions");
    if (!std::isfinite(charge)) QED_FAIL(QED_ERR_INVALID_ARG, "charge must be finite");
    if (!std::isfinite(dt) || dt < 0) QED_FAIL(QED_ERR_INVALID_ARG, "dt must be finite and >= 0");
    cudaStream_t st = as_stream(stream);
    if (prec == QED_F32)
        push_stored_kernel<float><<<resident_grid<push_stored_kernel<float>>(256, 0, sp->capacity), 256, 0, st>>>(
            push_seg<float>(sp, charge), dt);
    else
        push_stored_kernel<double><<<resident_grid<push_stored_kernel<double>>(256, 0, sp->capacity), 256, 0, st>>>(
            push_seg<double>(sp, charge), dt);
    QED_LAUNCH_CHECK();
    return QED_OK;
}
