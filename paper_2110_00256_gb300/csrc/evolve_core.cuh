// evolve_core.cuh -- the per-particle optical-depth evolution (chi, rate
// lookup, decrement, warp-ballot compaction of the firing particles) on values
// already in registers, and the 16-byte vector loads/stores of the particle
// arrays; shared by the evolution kernels and the fused push + evolution.
#pragma once

#include "evolve.cuh"
#include "physics.cuh"

namespace qed {

template <typename T, int VEC>
struct Vec;
template <>
struct Vec<float, 4> {
    using type = float4;
};
template <>
struct Vec<float, 2> {
    using type = float2;
};
template <>
struct Vec<double, 2> {
    using type = double2;
};

template <typename T, int VEC>
__device__ __forceinline__ void load_vec(const T *p, int64_t i, T (&out)[VEC])
{
    if constexpr (VEC == 1) {
        out[0] = __ldcs(p + i);
    } else {
        using V = typename Vec<T, VEC>::type;
        const V v = __ldcs(reinterpret_cast<const V *>(p + i));
        if constexpr (VEC == 4) {
            out[0] = v.x, out[1] = v.y, out[2] = v.z, out[3] = v.w;
        } else {
            out[0] = v.x, out[1] = v.y;
        }
    }
}

template <typename T, int VEC>
__device__ __forceinline__ void store_vec(T *p, int64_t i, const T (&in)[VEC])
{
    if constexpr (VEC == 1) {
        __stcs(p + i, in[0]);
    } else {
        using V = typename Vec<T, VEC>::type;
        V v;
        if constexpr (VEC == 4) {
            v.x = in[0], v.y = in[1], v.z = in[2], v.w = in[3];
        } else {
            v.x = in[0], v.y = in[1];
        }
        __stcs(reinterpret_cast<V *>(p + i), v);
    }
}

// one particle: chi, rate, optical-depth decrement; returns fire
template <typename T>
__device__ __forceinline__ bool evolve_one(int proc, const T *s_qs, const T *s_bw, const TablesView<T> &tv,
                                           T px, T py, T pz, T ex, T ey, T ez, T bx, T by, T bz, T dt, T cut,
                                           T &tau, T &tc, T &chi_out, int &bad)
{
    T chi, rate;
    if (proc == QED_PROC_QS) {
        T gamma, inv;
        chi = chi_lepton(px, py, pz, ex, ey, ez, bx, by, bz, gamma, inv);
        rate = qs_rate(s_qs, tv.qs_G, chi, gamma, inv);
    } else {
        T pm, inv;
        chi = chi_photon(px, py, pz, ex, ey, ez, bx, by, bz, pm, inv);
        rate = bw_rate(s_bw, tv.bw_T, chi, pm, inv);
    }
    const bool ok = isfinite(chi) && !isnan(tau) && isfinite(rate);
    bad += ok ? 0 : 1;
    if (!ok || chi < cut) rate = T(0);  // below the process's chi threshold: no evolution
    chi_out = chi;
    if constexpr (sizeof(T) == 4) {
        // Kahan-compensated decrement; tau - tc is the optical depth
        if (!isfinite(tau)) return false;  // removed particle (tau = +inf)
        const T y = d_fma(-rate, dt, -tc);
        const T t = tau + y;
        tc = (t - tau) - y;
        tau = t;
        return ok && (t < T(0) || (t == T(0) && tc > T(0)));
    } else {
        tau = tau - rate * dt;
        return ok && tau < T(0);
    }
}

// warp-ballot compaction of the firing particles among [i0, i0 + VEC) (cnt of
// them in this thread) into the segment's firing list: one atomic per warp
template <typename T, int VEC>
__device__ __forceinline__ void compact_fire(const EvolveSeg<T> &sg, int64_t i0, const bool (&fire)[VEC],
                                             const T (&chi)[VEC], int cnt, long long *stats)
{
    if (!__ballot_sync(0xffffffffu, cnt > 0)) return;
    const unsigned lane = threadIdx.x & 31u;
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o) incl += v;
    }
    const int wtot = __shfl_sync(0xffffffffu, incl, 31);
    unsigned long long base = 0;
    if (lane == 31) base = atomicAdd(sg.fire_count, (unsigned long long)wtot);
    base = __shfl_sync(0xffffffffu, base, 31);
    long long pos = (long long)base + incl - cnt;
    int over = 0;
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
        if (fire[j]) {
            if (pos < sg.fire_cap) {
                sg.fire_idx[pos] = i0 + j;
                sg.fire_chi[pos] = (double)chi[j];
            } else {
                ++over;
            }
            ++pos;
        }
    }
    warp_count_err(stats ? stats + QED_STAT_FIRE_OVERFLOW : nullptr, over, QED_EW_FIRE_OVERFLOW);
}

// Evaluate, store and compact VEC particles [i0, i0 + VEC) of segment `sg`
// whose inputs are already in registers (full: all VEC are live).  dry != 0
// evaluates everything but stores nothing (used by the launch-shape tuner).
template <typename T, int VEC>
__device__ __forceinline__ void evolve_regs(const EvolveSeg<T> &sg, int64_t n, int64_t i0, bool full,
                                            const T (&px)[VEC], const T (&py)[VEC], const T (&pz)[VEC],
                                            const T (&ex)[VEC], const T (&ey)[VEC], const T (&ez)[VEC],
                                            const T (&bx)[VEC], const T (&by)[VEC], const T (&bz)[VEC], T (&tau)[VEC],
                                            T (&tc)[VEC], const T *s_qs, const T *s_bw, const TablesView<T> &tab,
                                            T dt, T cut, long long *stats, int dry, int &bad)
{
    bool fire[VEC];
    T chi[VEC];
    int cnt = 0;
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
        T c = sizeof(T) == 4 ? tc[j] : T(0);
        fire[j] = evolve_one<T>(sg.proc, s_qs, s_bw, tab, px[j], py[j], pz[j], ex[j], ey[j], ez[j], bx[j], by[j],
                                bz[j], dt, cut, tau[j], c, chi[j], bad);
        tc[j] = c;
        fire[j] = fire[j] && (i0 + j < n);
        cnt += fire[j] ? 1 : 0;
    }
    if (dry) return;

    if (full) {
        store_vec<T, VEC>(sg.tau, i0, tau);
        if constexpr (sizeof(T) == 4) store_vec<T, VEC>(sg.tau_c, i0, tc);
    } else {
#pragma unroll
        for (int j = 0; j < VEC; ++j) {
            if (i0 + j < n) {
                sg.tau[i0 + j] = tau[j];
                if constexpr (sizeof(T) == 4) sg.tau_c[i0 + j] = tc[j];
            }
        }
    }

    compact_fire<T, VEC>(sg, i0, fire, chi, cnt, stats);
}

// scalar loads of the live particles among [i0, i0 + VEC) (ragged tail, misaligned arrays)
template <typename T, int VEC>
__device__ __forceinline__ void load_scalar(const EvolveSeg<T> &sg, int64_t n, int64_t i0, T (&px)[VEC],
                                            T (&py)[VEC], T (&pz)[VEC], T (&ex)[VEC], T (&ey)[VEC], T (&ez)[VEC],
                                            T (&bx)[VEC], T (&by)[VEC], T (&bz)[VEC], T (&tau)[VEC], T (&tc)[VEC])
{
#pragma unroll
    for (int j = 0; j < VEC; ++j) {
        const int64_t i = i0 + j;
        const bool v = i < n;
        px[j] = v ? sg.px[i] : T(0);
        py[j] = v ? sg.py[i] : T(0);
        pz[j] = v ? sg.pz[i] : T(0);
        ex[j] = v ? sg.ex[i] : T(0);
        ey[j] = v ? sg.ey[i] : T(0);
        ez[j] = v ? sg.ez[i] : T(0);
        bx[j] = v ? sg.bx[i] : T(0);
        by[j] = v ? sg.by[i] : T(0);
        bz[j] = v ? sg.bz[i] : T(0);
        tau[j] = v ? sg.tau[i] : T(1);
        tc[j] = (sizeof(T) == 4 && v) ? sg.tau_c[i] : T(0);
    }
}

// Segments in device memory (many patches): every CTA reads all segment
// counts (clamped to capacity) into s_n, forms the inclusive prefix of their
// tile counts in s_end by a block scan (thread k owns segments [k per,
// (k+1) per)), and returns the total number of tiles.  Ends with a barrier.
template <typename T, int THREADS>
__device__ __forceinline__ long long tile_prefix(const EvolveSeg<T> *__restrict__ segs, int n_seg, int64_t tile,
                                                 long long *s_end, long long *s_n, long long *s_warp)
{
    const int per = (n_seg + THREADS - 1) / THREADS;
    const int s0 = threadIdx.x * per, s1 = min(n_seg, s0 + per);
    long long local = 0;
    for (int s = s0; s < s1; ++s) {
        long long n = *segs[s].count;
        n = n < 0 ? 0 : (n > segs[s].capacity ? segs[s].capacity : n);
        s_n[s] = n;
        local += (n + tile - 1) / tile;
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
    long long woff = 0;
    for (int w = 0; w < warp; ++w) woff += s_warp[w];
    long long acc = woff + incl - local;
    for (int s = s0; s < s1; ++s) {
        acc += (s_n[s] + tile - 1) / tile;
        s_end[s] = acc;
    }
    __syncthreads();
    return n_seg ? s_end[n_seg - 1] : 0;
}

// the segment of tile t: the first s with s_end[s] > t
__device__ __forceinline__ int find_segment(const long long *s_end, int n_seg, long long t)
{
    int lo = 0, hi = n_seg - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (s_end[mid] > t)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

}  // namespace qed
