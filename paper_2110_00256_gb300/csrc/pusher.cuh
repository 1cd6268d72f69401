// pusher.cuh -- descriptors of the plane-wave particle push (see pusher.cu).
#pragma once

#include "common.cuh"

namespace qed {

struct WaveParams {
    double e0, omega, phase0;
    int circular, direction;
};

template <typename T>
struct PushSeg {
    T *x, *y, *z, *px, *py, *pz, *ex, *ey, *ez, *bx, *by, *bz;
    const int64_t *count;
    int64_t cap;
    T q;
};

template <typename T>
PushSeg<T> push_seg(const qed_species *s, double q);

template <typename T>
qed_status launch_push(const void *d_segs, int n_seg, const WaveParams &w, double t0, double dt,
                       const int64_t *d_step, int64_t step, int64_t capacity, cudaStream_t st);

qed_status check_wave(const qed_plane_wave *w);
WaveParams wave_params(const qed_plane_wave *w);

}  // namespace qed
