// pusher.cuh -- descriptors and per-particle arithmetic of the particle push
// (see pusher.cu); the fused push + evolution uses the same functions.
#pragma once

#include "common.cuh"
#include "evolve.cuh"

namespace qed {

struct WaveParams {
    double e0, omega_pi, phase0_pi;  // amplitude; omega / pi and phase0 / pi (phases in half-turns)
    int circular, direction;
};

template <typename T>
struct PushSeg {
    T *x, *y, *z, *px, *py, *pz, *ex, *ey, *ez, *bx, *by, *bz;
    const int64_t *count;
    int64_t cap;
    T q;
};

// sin and cos of pi u (the argument reduction of a half-turn multiple is exact)
__device__ __forceinline__ void d_sincospi(float u, float *s, float *c) { sincospif(u, s, c); }
__device__ __forceinline__ void d_sincospi(double u, double *s, double *c) { sincospi(u, s, c); }

// the wave's parameters and the time in the working precision, converted once
// per thread (conversions from FP64 run on GB300's narrow FP64 pipe)
template <typename T>
struct WaveT {
    T omega_pi, phase0_pi, e0, d, t;
    int circular;
};

template <typename T>
__device__ __forceinline__ WaveT<T> wave_at(const WaveParams &w, double t)
{
    return WaveT<T>{(T)w.omega_pi, (T)w.phase0_pi, (T)w.e0, (T)w.direction, (T)t, w.circular};
}

// phase phi = omega (t - d x) + phase0; E = E0 (0, cos phi, [sin phi]); B = d x-hat cross E.
// Evaluated in the working precision, in half-turns (over the cascade's 10
// periods the FP32 phase keeps ~1e-5 rad).
template <typename T>
__device__ __forceinline__ void wave_fields(const WaveT<T> &w, T x, T &ex, T &ey, T &ez, T &bx, T &by, T &bz)
{
    const T u = w.omega_pi * (w.t - w.d * x) + w.phase0_pi;
    T s, c;
    d_sincospi(u, &s, &c);
    ex = T(0);
    ey = w.e0 * c;
    ez = w.circular ? w.e0 * s : T(0);
    bx = T(0);
    by = -w.d * ez;
    bz = w.d * ey;
}

// reciprocal square root: FP32 rsqrtf (within 2 ulp), FP64 rsqrt (within 1 ulp);
// the push is not part of the paper's method, and its arithmetic budget is the
// fused cascade kernel's limit
__device__ __forceinline__ float d_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double d_rsqrt(double x) { return rsqrt(x); }

// one step of the momentum of a particle of charge q (relativistic Boris
// rotation; q = 0: a photon, unchanged) and the velocity it then moves with
template <typename T>
__device__ __forceinline__ void boris_move(T q, T dt, T ex, T ey, T ez, T bx, T by, T bz, T &px, T &py, T &pz,
                                           T &vx, T &vy, T &vz)
{
    if (q == T(0)) {
        const T p2 = px * px + py * py + pz * pz;
        const T inv = p2 > T(0) ? d_rsqrt(p2) : T(0);
        vx = px * inv, vy = py * inv, vz = pz * inv;
        return;
    }
    const T h = T(0.5) * q * dt;
    const T mx = px + h * ex, my = py + h * ey, mz = pz + h * ez;  // half electric kick
    const T hg = h * d_rsqrt(T(1) + mx * mx + my * my + mz * mz);
    const T tx = hg * bx, ty = hg * by, tz = hg * bz;
    const T f = T(2) / (T(1) + tx * tx + ty * ty + tz * tz);
    const T sx = f * tx, sy = f * ty, sz = f * tz;
    const T qx = mx + (my * tz - mz * ty), qy = my + (mz * tx - mx * tz), qz = mz + (mx * ty - my * tx);
    px = mx + (qy * sz - qz * sy) + h * ex;
    py = my + (qz * sx - qx * sz) + h * ey;
    pz = mz + (qx * sy - qy * sx) + h * ez;
    const T ig = d_rsqrt(T(1) + px * px + py * py + pz * pz);
    vx = px * ig, vy = py * ig, vz = pz * ig;
}

template <typename T>
PushSeg<T> push_seg(const qed_species *s, double q);

template <typename T>
qed_status launch_push(const void *d_segs, int n_seg, const WaveParams &w, double t0, double dt,
                       const int64_t *d_step, int64_t step, int64_t capacity, cudaStream_t st);

// the fused push + evolution over segments in device memory (fused.cu): d_push
// holds PushSeg<T>[n_seg] in the order of d_segs; store_fields != 0 also writes
// the fields into the species; vec: every array 16-byte aligned
template <typename T>
qed_status launch_push_evolve(const EvolveSeg<T> *d_segs, const void *d_push, int n_seg, const TablesView<T> &tab,
                              const WaveParams &w, double t0, double dt, const int64_t *d_step, int64_t step,
                              T cut_qs, T cut_bw, long long *stats, int store_fields, bool vec, cudaStream_t st);

qed_status check_wave(const qed_plane_wave *w);
WaveParams wave_params(const qed_plane_wave *w);

}  // namespace qed
