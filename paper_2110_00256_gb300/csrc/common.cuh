// common.cuh -- shared device/host helpers of libqed (GB300, sm_103a).
//
// Status handling for the C ABI, the Philox4x32-10 counter-based generator
// (Salmon, Moraes, Dror, Shaw, SC'11), the device views of the lookup tables,
// and warp-aggregated append/counter helpers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <string>

#include "qed.h"

namespace qed {

// ---------------------------------------------------------------------------
// status / error messages (thread-local, see qed_last_error_message)
// ---------------------------------------------------------------------------
void set_error(const char *fmt, ...);
void clear_error();

#define QED_FAIL(code, ...)          \
    do {                             \
        ::qed::set_error(__VA_ARGS__); \
        return (code);               \
    } while (0)

#define QED_CUDA_TRY(expr)                                                              \
    do {                                                                                \
        cudaError_t _e = (expr);                                                        \
        if (_e != cudaSuccess)                                                          \
            QED_FAIL(QED_ERR_CUDA, "%s failed: %s (%s:%d)", #expr, cudaGetErrorString(_e), \
                     __FILE__, __LINE__);                                               \
    } while (0)

#define QED_LAUNCH_CHECK()                                                               \
    do {                                                                                 \
        cudaError_t _e = cudaGetLastError();                                             \
        if (_e != cudaSuccess)                                                           \
            QED_FAIL(QED_ERR_CUDA, "kernel launch failed: %s (%s:%d)", cudaGetErrorString(_e), \
                     __FILE__, __LINE__);                                                \
    } while (0)

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// 64-bit FNV-1a of a byte range (the checksum of the table and network files)
inline uint64_t fnv1a64(const void *data, size_t n)
{
    const unsigned char *b = (const unsigned char *)data;
    uint64_t h = 0xcbf29ce484222325ull;
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 0x100000001b3ull;
    }
    return h;
}

// fine-structure constant, CODATA 2018 (the paper prints no value)
constexpr double kAlpha = 7.2973525693e-3;

// ---------------------------------------------------------------------------
// Philox4x32-10: ten rounds of two 32x32 -> 64-bit products, Weyl key bumps.
// counter = (id_lo, id_hi, step, purpose), key = (seed_lo, seed_hi).
// ---------------------------------------------------------------------------
enum Purpose : uint32_t { kSample = 0, kTauReset = 1, kTauInit = 2, kChildId = 3 };

struct U4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                       uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t a = 0xD2511F53u * c0, ah = __umulhi(0xD2511F53u, c0);
        const uint32_t b = 0xCD9E8D57u * c2, bh = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = bh ^ c1 ^ k0;
        const uint32_t n2 = ah ^ c3 ^ k1;
        c0 = n0;
        c1 = b;
        c2 = n2;
        c3 = a;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return U4{c0, c1, c2, c3};
}

__device__ __forceinline__ U4 draw(uint64_t seed, uint64_t id, int64_t step, uint32_t purpose)
{
    return philox10((uint32_t)id, (uint32_t)(id >> 32), (uint32_t)(uint64_t)step, purpose,
                    (uint32_t)seed, (uint32_t)(seed >> 32));
}

// 53-bit uniform in (0, 1): ((lo | hi << 32) >> 11 + 1/2) * 2^-53
__device__ __forceinline__ double uniform53(uint32_t lo, uint32_t hi)
{
    const uint64_t v = (((uint64_t)hi << 32) | lo) >> 11;
    // ((double)v + 0.5) 2^-53 assembled from integer operations, bit for bit the
    // same double without an FP64 instruction: v + 1/2 is exact below 2^52 and
    // rounds to even above it, so U = M 2^-k with M = 2v + 1, k = 54 (v < 2^52)
    // or M = v + (v & 1), k = 53; M < 2^53 except M = 2^53 (U = 1)
    const bool big = v >= (1ull << 52);
    const uint64_t m = big ? v + (v & 1ull) : 2ull * v + 1ull;
    const int k = big ? 53 : 54;
    const int len = 64 - __clzll((long long)m);  // bit length, 1 .. 54
    const uint64_t frac = (len <= 53 ? m << (53 - len) : m >> 1) & 0xfffffffffffffull;
    return __longlong_as_double((long long)(((uint64_t)(len - 1 - k + 1023) << 52) | frac));
}

// ---------------------------------------------------------------------------
// device views of the tables (non-owning, passed by value to kernels)
// ---------------------------------------------------------------------------
template <typename T>
struct Table1D {
    const T *ln_f;   // [n]
    T ln_min;        // ln chi_min
    T inv_d;         // (n - 1) / (ln chi_max - ln chi_min)
    T chi_min, chi_max;
    int n;
};

// bins of the guide tables that bracket the inverse-CDF search
constexpr int kGuideBins = 64;

template <typename T>
struct Table2D {
    const T *v;      // [n_chi][n_xi], ln P (QS) or P (BW)
    const T *dv;     // [n_chi][n_xi], v[n][m+1] - v[n][m] formed in FP64 (last column 0)
    const int32_t *guide;  // [n_chi][kGuideBins + 1]: per row, the largest m with v[n][m] at or
                           // below each edge of kGuideBins equal bins of the uniform draw r
    T ln_min, inv_d, chi_min, chi_max;
    T x0, dx;        // xi axis: QS ln xi_min and step in ln xi; BW 0 and step in xi
    int n_chi, n_xi;
};

template <typename T>
struct TablesView {
    Table1D<T> qs_G, bw_T;
    Table2D<T> qs_P, bw_P;
};

// ---------------------------------------------------------------------------
// warp helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// Reserve `want` (0/1) slots per lane from *counter with one atomic per warp;
// all 32 lanes must call it.  Returns the slot of this lane (valid iff want).
__device__ __forceinline__ long long warp_reserve(unsigned long long *counter, bool want)
{
    const unsigned m = __ballot_sync(0xffffffffu, want);
    long long base = 0;
    if (m) {
        const int leader = __ffs(m) - 1;
        if ((int)lane_id() == leader) base = (long long)atomicAdd(counter, (unsigned long long)__popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
    }
    return base + __popc(m & ((1u << lane_id()) - 1u));
}

// Add per-lane counts to a 64-bit device counter with one atomic per warp.
__device__ __forceinline__ void warp_count(long long *ctr, int v)
{
    if (ctr == nullptr) return;
    int s = v;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane_id() == 0 && s) atomicAdd((unsigned long long *)ctr, (unsigned long long)s);
}

// ---------------------------------------------------------------------------
// device error word (qed_device_status): every translation unit keeps its own
// word, which its kernels OR their QED_EW_* bits into whether or not the caller
// passed a statistics array; a host-side registry reads (and clears) all of them.
// ---------------------------------------------------------------------------
static __device__ unsigned int g_err_word;

__device__ __forceinline__ void note_error(unsigned bit) { atomicOr(&g_err_word, bit); }

// per-lane counts into a statistic (if any) and, where a lane counted, the error bit
__device__ __forceinline__ void warp_count_err(long long *ctr, int v, unsigned bit)
{
    if (v) note_error(bit);
    warp_count(ctr, v);
}

using ErrWordIO = cudaError_t (*)(unsigned *out, bool clear);
int register_err_word(ErrWordIO f);

static cudaError_t err_word_io(unsigned *out, bool clear)
{
    cudaError_t e = cudaMemcpyFromSymbol(out, g_err_word, sizeof(unsigned));
    if (e == cudaSuccess && clear) {
        const unsigned z = 0;
        e = cudaMemcpyToSymbol(g_err_word, &z, sizeof(unsigned));
    }
    return e;
}

[[maybe_unused]] static const int g_err_word_registered = register_err_word(&err_word_io);

}  // namespace qed

// opaque handle definition shared by the .cu files
struct qed_tables {
    qed_table_params params;
    int device;
    double *d_qs_lnG, *d_qs_lnP, *d_bw_lnT, *d_bw_P;  // FP64
    float *f_qs_lnG, *f_qs_lnP, *f_bw_lnT, *f_bw_P;   // FP32 copies (round to nearest)
    // column differences of the 2-D tables, formed in FP64 (then rounded for the
    // FP32 copies): the slope of the inverse-CDF interpolation keeps its relative
    // accuracy even where neighbouring table entries are close
    double *d_qs_dlnP, *d_bw_dP;
    float *f_qs_dlnP, *f_bw_dP;
    // guide tables of the 2-D tables' inverse-CDF search, one per precision
    int32_t *d_qs_guide, *d_bw_guide, *f_qs_guide, *f_bw_guide;
};

namespace qed {
template <typename T>
TablesView<T> make_view(const qed_tables *t);
qed_status check_tables(const qed_tables *t);
qed_status check_species(const qed_species *s, const char *name, qed_precision prec);
}  // namespace qed
