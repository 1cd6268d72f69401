// upkeep.cu -- per-species energy sums (the quantity that photon emission and
// pair production conserve, §2.1, §2.2) and the compaction of removed
// particles (the photons that pair production consumed, §3.1), so that they
// stop being read every step.
#include "launch.cuh"

namespace qed {

// ---------------------------------------------------------------------------
// energy: sum of w * gamma (leptons) or w * |p| (photons), FP64
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) energy_kernel(const T *__restrict__ px, const T *__restrict__ py,
                                                     const T *__restrict__ pz, const T *__restrict__ w,
                                                     const int64_t *count, int64_t capacity, int photon, double *out)
{
    __shared__ double s_e[8], s_c[8];
    int64_t n = *count;
    n = n < 0 ? 0 : (n > capacity ? capacity : n);
    double e = 0.0, c = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = px[i], y = py[i], z = pz[i], ww = w[i];
        const double p2 = x * x + y * y + z * z;
        e += ww * sqrt(photon ? p2 : 1.0 + p2);
        c += ww != 0.0 ? 1.0 : 0.0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_xor_sync(0xffffffffu, e, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    const int warp = threadIdx.x >> 5;
    if (lane_id() == 0) s_e[warp] = e, s_c[warp] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        double se = 0.0, sc = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) se += s_e[k], sc += s_c[k];
        if (se != 0.0) atomicAdd(out, se);
        if (sc != 0.0) atomicAdd(out + 1, sc);
    }
}

// ---------------------------------------------------------------------------
// compaction.  work layout (int64): [0] r = removed among [0, n), [1] n' = n - r,
// [2] H = removed among [0, n') (= live among [n', n)), [3] n, [4..8) unused,
// [8, 8 + tiles) per-tile removed counts, then exclusive offsets in place,
// then holes[capacity], movers[capacity].
// ---------------------------------------------------------------------------
constexpr int kCompactThreads = 256;
constexpr int kCompactItems = 8;
constexpr int64_t kCompactTile = (int64_t)kCompactThreads * kCompactItems;  // 2048, as QED_COMPACT_WORK assumes

template <typename T>
struct CompactView {
    T *f[9];      // px .. bz
    T *tau, *tau_c, *w;
    T *pos[3];    // x, y, z or NULL
    uint64_t *id;
    int64_t *count;
    int64_t capacity;
};

template <typename T>
__device__ __forceinline__ bool is_removed(const CompactView<T> &v, int64_t i)
{
    const T t = v.tau[i];
    return v.w[i] == T(0) && isinf(t) && t > T(0);
}

__device__ __forceinline__ int64_t clamp_count(const int64_t *count, int64_t capacity)
{
    const int64_t n = *count;
    return n < 0 ? 0 : (n > capacity ? capacity : n);
}

// per-tile counts of removed particles
template <typename T>
__global__ void __launch_bounds__(kCompactThreads) compact_count_kernel(CompactView<T> v, int64_t *work)
{
    __shared__ int s_w[kCompactThreads / 32];
    const int64_t n = clamp_count(v.count, v.capacity);
    const int64_t tiles = (n + kCompactTile - 1) / kCompactTile;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        int c = 0;
        for (int k = 0; k < kCompactItems; ++k) {
            const int64_t i = t * kCompactTile + (int64_t)k * kCompactThreads + threadIdx.x;
            c += (i < n && is_removed(v, i)) ? 1 : 0;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane_id() == 0) s_w[threadIdx.x >> 5] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
            int s = 0;
            for (int k = 0; k < kCompactThreads / 32; ++k) s += s_w[k];
            work[8 + t] = s;
        }
        __syncthreads();
    }
}

// one CTA: exclusive scan of the tile counts, r, n', and H (the removed ones
// before n', counted in n''s tile directly)
template <typename T>
__global__ void __launch_bounds__(1024) compact_scan_kernel(CompactView<T> v, int64_t *work, long long *stats)
{
    __shared__ long long s_part[1024];
    __shared__ long long s_h[32];
    const int64_t n = clamp_count(v.count, v.capacity);
    const int64_t tiles = (n + kCompactTile - 1) / kCompactTile;
    const int64_t per = (tiles + 1023) / 1024;
    const int64_t a = threadIdx.x * per, b = min(tiles, a + per);
    long long sum = 0;
    for (int64_t t = a; t < b; ++t) sum += work[8 + t];
    s_part[threadIdx.x] = sum;
    __syncthreads();
    // Hillis-Steele inclusive scan of the 1024 partial sums
    for (int o = 1; o < 1024; o <<= 1) {
        const long long add = threadIdx.x >= o ? s_part[threadIdx.x - o] : 0;
        __syncthreads();
        s_part[threadIdx.x] += add;
        __syncthreads();
    }
    long long off = s_part[threadIdx.x] - sum;
    for (int64_t t = a; t < b; ++t) {
        const long long c = work[8 + t];
        work[8 + t] = off;
        off += c;
    }
    const long long r = s_part[1023];
    const int64_t np = n - r;
    __syncthreads();
    // H = offset of n''s tile + removed in [tile start, n')
    const int64_t tn = np / kCompactTile;
    const int64_t lo = tn * kCompactTile;
    int c = 0;
    for (int64_t i = lo + threadIdx.x; i < np; i += 1024) c += is_removed(v, i) ? 1 : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane_id() == 0) s_h[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long h = tn < tiles ? work[8 + tn] : r;
        if (tn < tiles)
            for (int k = 0; k < 32; ++k) h += s_h[k];
        work[0] = r;
        work[1] = np;
        work[2] = h;
        work[3] = n;
        if (stats && r) atomicAdd((unsigned long long *)(stats + QED_STAT_COMPACTED), (unsigned long long)r);
    }
}

// holes[R(i)] = i for removed i < n'; movers[L(i) - (n' - H)] = i for live i >= n'
// (R, L: removed / live particles before i)
template <typename T>
__global__ void __launch_bounds__(kCompactThreads) compact_list_kernel(CompactView<T> v, int64_t *work)
{
    __shared__ int s_w[kCompactThreads / 32];
    const int64_t n = work[3], np = work[1], H = work[2];
    if (H == 0) return;
    const int64_t tiles = (n + kCompactTile - 1) / kCompactTile;
    int64_t *holes = work + 8 + (v.capacity + kCompactTile - 1) / kCompactTile;
    int64_t *movers = holes + v.capacity;
    const int lane = lane_id(), warp = threadIdx.x >> 5;
    for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
        // thread k owns the kCompactItems consecutive particles [t T + k I, t T + (k + 1) I)
        const int64_t i0 = t * kCompactTile + (int64_t)threadIdx.x * kCompactItems;
        bool rm[kCompactItems];
        int c = 0;
#pragma unroll
        for (int k = 0; k < kCompactItems; ++k) {
            rm[k] = (i0 + k < n) && is_removed(v, i0 + k);
            c += rm[k] ? 1 : 0;
        }
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int x = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += x;
        }
        if (lane == 31) s_w[warp] = incl;
        __syncthreads();
        int woff = 0;
        for (int k = 0; k < warp; ++k) woff += s_w[k];
        long long R = work[8 + t] + woff + incl - c;  // removed before i0
#pragma unroll
        for (int k = 0; k < kCompactItems; ++k) {
            const int64_t i = i0 + k;
            if (i < n) {
                if (rm[k]) {
                    if (i < np) holes[R] = i;
                    ++R;
                } else if (i >= np) {
                    movers[(i - R) - (np - H)] = i;
                }
            }
        }
        __syncthreads();
    }
}

// move movers[k] -> holes[k] for k < H, every array; then the count becomes n'
template <typename T>
__global__ void __launch_bounds__(256) compact_move_kernel(CompactView<T> v, int64_t *work)
{
    const int64_t np = work[1], H = work[2];
    const int64_t *holes = work + 8 + (v.capacity + kCompactTile - 1) / kCompactTile;
    const int64_t *movers = holes + v.capacity;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < H; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = movers[k], d = holes[k];
#pragma unroll
        for (int a = 0; a < 9; ++a) v.f[a][d] = v.f[a][s];
        v.tau[d] = v.tau[s];
        if (v.tau_c) v.tau_c[d] = v.tau_c[s];
        v.w[d] = v.w[s];
        v.id[d] = v.id[s];
#pragma unroll
        for (int a = 0; a < 3; ++a)
            if (v.pos[a]) v.pos[a][d] = v.pos[a][s];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *v.count = np;
}

template <typename T>
static qed_status compact_impl(const qed_species *sp, int64_t *work, long long *stats, cudaStream_t st)
{
    CompactView<T> v;
    void *const f[9] = {sp->px, sp->py, sp->pz, sp->ex, sp->ey, sp->ez, sp->bx, sp->by, sp->bz};
    for (int a = 0; a < 9; ++a) v.f[a] = (T *)f[a];
    v.tau = (T *)sp->tau;
    v.tau_c = sizeof(T) == 4 ? (T *)sp->tau_c : nullptr;
    v.w = (T *)sp->weight;
    v.pos[0] = (T *)sp->x, v.pos[1] = (T *)sp->y, v.pos[2] = (T *)sp->z;
    v.id = sp->id;
    v.count = sp->d_count;
    v.capacity = sp->capacity;
    const int64_t tiles = (sp->capacity + kCompactTile - 1) / kCompactTile;
    const int gc = resident_grid<compact_count_kernel<T>>(kCompactThreads, 0, tiles * kCompactThreads);
    compact_count_kernel<T><<<gc, kCompactThreads, 0, st>>>(v, work);
    compact_scan_kernel<T><<<1, 1024, 0, st>>>(v, work, stats);
    const int gl = resident_grid<compact_list_kernel<T>>(kCompactThreads, 0, tiles * kCompactThreads);
    compact_list_kernel<T><<<gl, kCompactThreads, 0, st>>>(v, work);
    const int gm = resident_grid<compact_move_kernel<T>>(256, 0, sp->capacity);
    compact_move_kernel<T><<<gm, 256, 0, st>>>(v, work);
    QED_LAUNCH_CHECK();
    return QED_OK;
}

}  // namespace qed

using namespace qed;

extern "C" qed_status qed_species_energy(const qed_species *sp, qed_precision prec, int32_t photon, double *d_out,
                                         void *stream)
{
    clear_error();
    qed_status s = check_species(sp, "species", prec);
    if (s) return s;
    if (d_out == nullptr || ((uintptr_t)d_out & 7u)) QED_FAIL(QED_ERR_INVALID_ARG, "d_out is NULL or misaligned");
    cudaStream_t st = as_stream(stream);
    if (prec == QED_F32) {
        const int g = resident_grid<energy_kernel<float>>(256, 0, sp->capacity);
        energy_kernel<float><<<g, 256, 0, st>>>((const float *)sp->px, (const float *)sp->py, (const float *)sp->pz,
                                                (const float *)sp->weight, sp->d_count, sp->capacity, photon != 0,
                                                d_out);
    } else {
        const int g = resident_grid<energy_kernel<double>>(256, 0, sp->capacity);
        energy_kernel<double><<<g, 256, 0, st>>>((const double *)sp->px, (const double *)sp->py,
                                                 (const double *)sp->pz, (const double *)sp->weight, sp->d_count,
                                                 sp->capacity, photon != 0, d_out);
    }
    QED_LAUNCH_CHECK();
    return QED_OK;
}

extern "C" qed_status qed_compact_species(const qed_species *sp, qed_precision prec, int64_t *d_work,
                                          int64_t work_capacity, int64_t *d_stats, void *stream)
{
    clear_error();
    qed_status s = check_species(sp, "species", prec);
    if (s) return s;
    if (d_work == nullptr || ((uintptr_t)d_work & 7u)) QED_FAIL(QED_ERR_INVALID_ARG, "d_work is NULL or misaligned");
    const int64_t need = QED_COMPACT_WORK(sp->capacity);
    if (work_capacity < need)
        QED_FAIL(QED_ERR_INVALID_ARG, "d_work holds %lld entries, %lld needed for capacity %lld",
                 (long long)work_capacity, (long long)need, (long long)sp->capacity);
    if ((sp->x == nullptr) != (sp->y == nullptr) || (sp->x == nullptr) != (sp->z == nullptr))
        QED_FAIL(QED_ERR_INVALID_ARG, "positions must be all set or all NULL");
    cudaStream_t st = as_stream(stream);
    return prec == QED_F32 ? compact_impl<float>(sp, d_work, (long long *)d_stats, st)
                           : compact_impl<double>(sp, d_work, (long long *)d_stats, st);
}
