// evolve.cuh -- launch descriptors of the batched optical-depth evolution.
#pragma once

#include <cmath>
#include <cstring>

#include "common.cuh"

namespace qed {

constexpr int kEvolveThreads = 256;
template <typename T, int VEC>
constexpr int64_t kEvolveTile = (int64_t)kEvolveThreads * VEC;

template <typename T>
struct EvolveSeg {
    const T *px, *py, *pz, *ex, *ey, *ez, *bx, *by, *bz;
    T *tau, *tau_c;
    const int64_t *count;
    int64_t capacity;
    int64_t *fire_idx;
    double *fire_chi;
    unsigned long long *fire_count;
    int64_t fire_cap;
    int proc;
};

template <typename T, int MAXSEG>
struct EvolveArgs {
    EvolveSeg<T> seg[MAXSEG];
    TablesView<T> tab;
    long long *stats;
    long long wait_cycles;  // limit of the producer/consumer waits of the bulk-copy form (0: kWaitCycles)
    T dt;
    T chi_cut[2];  // per process (QED_PROC_QS, QED_PROC_BW): below it the rate is taken as zero
    int n_seg;
};

int sm_count();

// pipeline: QED_EVOLVE_* (the bulk-copy pipeline applies to FP32 with
// 16-byte-aligned arrays; threads 512 or ctas_per_sm 2 pick its other shapes)
template <typename T, int MAXSEG>
qed_status launch_evolve(const EvolveArgs<T, MAXSEG> &a, bool vec_ok, int64_t capacity_sum, int grid_override,
                         cudaStream_t st, int pipeline = 0, int threads = 0, int ctas_per_sm = 0);

template <typename T>
bool fill_seg(EvolveSeg<T> &g, const qed_species *sp, int proc, const qed_fire_list *fire);

// segments in device memory (the batched substep); threads in {128, 256, 512},
// ctas_per_sm 0 = as many as the register budget allows; dry != 0 stores nothing;
// cut_qs / cut_bw: chi thresholds of the two processes (rate zero below)
template <typename T>
qed_status launch_evolve_segments(const EvolveSeg<T> *d_segs, int n_seg, const TablesView<T> &tab, T dt, T cut_qs,
                                  T cut_bw, long long *stats, int dry, bool vec, int threads, int ctas_per_sm,
                                  cudaStream_t st);

qed_status check_fire(const qed_fire_list *f, const char *name);

__global__ void clamp_fire_counts(unsigned long long *c0, int64_t cap0, unsigned long long *c1, int64_t cap1,
                                  unsigned long long *c2, int64_t cap2);

}  // namespace qed
