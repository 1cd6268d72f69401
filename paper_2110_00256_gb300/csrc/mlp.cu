// mlp.cu -- the learned sampler's object, training (forward + backward on the
// CUDA cores in FP32 with the same bf16 rounding as inference, Adam), batch
// inference with the 64x64 layer on the tcgen05 tensor cores, and batch
// sampling through the 2-D tables for comparison.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "launch.cuh"
#include "mlp.cuh"
#include "physics.cuh"
#include "tcgen05.cuh"

namespace qed {

MlpView mlp_view(const qed_mlp *m, int proc)
{
    MlpView v;
    v.w = m->w[proc];
    v.ln_min = (float)std::log(m->chi_min[proc]);
    v.ln_max = (float)std::log(m->chi_max[proc]);
    v.scale = (float)(2.0 / (std::log(m->chi_max[proc]) - std::log(m->chi_min[proc])));
    v.proc = proc;
    return v;
}

// ---------------------------------------------------------------------------
// initialisation: Glorot-uniform weights from Philox, zero biases
// ---------------------------------------------------------------------------
__global__ void mlp_init_kernel(float *p, uint64_t seed, int proc)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kMlpParams; i += gridDim.x * blockDim.x) {
        float a = 0.f;
        if (i < kOffB1)
            a = sqrtf(6.f / (2 + kMlpH));
        else if (i >= kOffW2 && i < kOffB2)
            a = sqrtf(6.f / (kMlpH + kMlpH));
        else if (i >= kOffW3 && i < kOffB3)
            a = sqrtf(6.f / (kMlpH + 1));
        const U4 w = draw(seed, (uint64_t)proc * 1000003ull + (uint64_t)i, 0, 5u);
        const float u = (float)uniform53(w.x, w.y);
        p[i] = a * (2.f * u - 1.f);
    }
}

__global__ void mlp_to_bf16_kernel(const float *p, __nv_bfloat16 *w)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kMlpParams; i += gridDim.x * blockDim.x)
        w[i] = __float2bfloat16_rn(p[i]);
}

// ---------------------------------------------------------------------------
// training: one CTA of kTrainThreads threads takes kTrainThreads samples at a
// time (one per thread) and accumulates the gradient of the mean squared error
// in shared memory; each CTA stores its sums (gradient and loss) in a slot of
// its own, and mlp_reduce_kernel adds the slots in CTA order, so that a
// training run gives the same bits every time (atomic adds across CTAs would
// round in the order the CTAs arrive).
// ---------------------------------------------------------------------------
constexpr int kTrainThreads = 128;
constexpr int kTS = kTrainThreads + 1;  // padded sample stride of the [64][samples] buffers

struct TrainSmem {
    alignas(8) float w1a[kMlpH];
    alignas(8) float w1b[kMlpH];
    alignas(8) float b1[kMlpH];
    float w2[kMlpH * kMlpH], b2[kMlpH], w3[kMlpH], b3;
    float g[kMlpParams];       // gradient accumulator of this CTA
    float h1[kMlpH * kTS];     // bf16-rounded h1, [k][s]
    float z2[kMlpH * kTS];     // z2, then d2 = dL/dz2
    float q[kMlpH * kTS];      // dy * h2, then d1 = dL/dz1
    float x[2][kTrainThreads], dy[kTrainThreads];
};

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__global__ void __launch_bounds__(kTrainThreads) mlp_train_kernel(MlpView v, const double *__restrict__ chi,
                                                                    const double *__restrict__ uu,
                                                                    const double *__restrict__ xi, int64_t n,
                                                                    float *part)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TrainSmem &S = *reinterpret_cast<TrainSmem *>(smem_raw);
    const int tid = threadIdx.x;
    for (int i = tid; i < kMlpH; i += blockDim.x) {
        S.w1a[i] = __bfloat162float(v.w[kOffW1 + 2 * i]);
        S.w1b[i] = __bfloat162float(v.w[kOffW1 + 2 * i + 1]);
    }
    for (int i = tid; i < kMlpH * kMlpH; i += blockDim.x) S.w2[i] = __bfloat162float(v.w[kOffW2 + i]);
    for (int i = tid; i < kMlpH; i += blockDim.x) {
        S.b1[i] = __bfloat162float(v.w[kOffB1 + i]);
        S.b2[i] = __bfloat162float(v.w[kOffB2 + i]);
        S.w3[i] = __bfloat162float(v.w[kOffW3 + i]);
    }
    for (int i = tid; i < kMlpParams; i += blockDim.x) S.g[i] = 0.f;
    if (tid == 0) S.b3 = __bfloat162float(v.w[kOffB3]);
    __syncthreads();
    const float inv_n = 1.0f / (float)n;
    float my_loss = 0.f;

    for (int64_t base = (int64_t)blockIdx.x * kTrainThreads; base < n; base += (int64_t)gridDim.x * kTrainThreads) {
        const int64_t i = base + tid;
        const bool valid = i < n;
        float x1 = 0.f, x2 = 0.f, tgt = 0.f;
        if (valid) {
            const MlpIn in = mlp_input(v, chi[i], uu[i]);
            x1 = in.x1, x2 = in.x2;
            tgt = mlp_target(v.proc, xi[i], in);
        }
        S.x[0][tid] = x1;
        S.x[1][tid] = x2;
        // forward, with the inference kernels' arithmetic (pairs of neurons)
        const uint64_t x1x1 = f2(x1, x1), x2x2 = f2(x2, x2);
        for (int k = 0; k < kMlpH; k += 2) {
            const float2 g = f2u(layer1_pair(S.w1a, S.w1b, S.b1, k, x1x1, x2x2));
            S.h1[k * kTS + tid] = bf16r(g.x);
            S.h1[(k + 1) * kTS + tid] = bf16r(g.y);
        }
        float y = S.b3;
        for (int j = 0; j < kMlpH; j += 2) {
            float z0 = S.b2[j], z1 = S.b2[j + 1];
            for (int k = 0; k < kMlpH; ++k) {
                const float h = S.h1[k * kTS + tid];
                z0 = fmaf(S.w2[j * kMlpH + k], h, z0);
                z1 = fmaf(S.w2[(j + 1) * kMlpH + k], h, z1);
            }
            S.z2[j * kTS + tid] = z0;
            S.z2[(j + 1) * kTS + tid] = z1;
            const float2 g = f2u(gelu2(f2(z0, z1)));
            S.q[j * kTS + tid] = g.x;
            S.q[(j + 1) * kTS + tid] = g.y;
            y = fmaf(S.w3[j + 1], g.y, fmaf(S.w3[j], g.x, y));
        }
        const float r = valid ? y - tgt : 0.f;
        my_loss += r * r;
        const float dy = 2.f * r * inv_n;
        S.dy[tid] = dy;
        for (int j = 0; j < kMlpH; ++j) {
            const float z = S.z2[j * kTS + tid];
            S.q[j * kTS + tid] *= dy;                             // dy h2, for dW3
            S.z2[j * kTS + tid] = dy * S.w3[j] * gelu_grad(z);    // d2
        }
        __syncthreads();
        // dW2 = d2^T h1, db2 = sum d2, dW3 = sum dy h2, db3 = sum dy
        for (int e = tid; e < kMlpH * kMlpH; e += blockDim.x) {
            const int j = e / kMlpH, k = e % kMlpH;
            float acc = 0.f;
            for (int s = 0; s < kTrainThreads; ++s) acc = fmaf(S.z2[j * kTS + s], S.h1[k * kTS + s], acc);
            S.g[kOffW2 + e] += acc;
        }
        if (tid < kMlpH) {
            float a = 0.f, b = 0.f;
            for (int s = 0; s < kTrainThreads; ++s) {
                a += S.z2[tid * kTS + s];
                b += S.q[tid * kTS + s];
            }
            S.g[kOffB2 + tid] += a;
            S.g[kOffW3 + tid] += b;
        } else if (tid == kMlpH) {
            float a = 0.f;
            for (int s = 0; s < kTrainThreads; ++s) a += S.dy[s];
            S.g[kOffB3] += a;
        }
        __syncthreads();
        // d1 = (W2^T d2) * gelu'(z1), per sample
        for (int k = 0; k < kMlpH; ++k) {
            float acc = 0.f;
            for (int j = 0; j < kMlpH; ++j) acc = fmaf(S.w2[j * kMlpH + k], S.z2[j * kTS + tid], acc);
            const float z1 = fmaf(S.w1a[k], x1, fmaf(S.w1b[k], x2, S.b1[k]));
            S.q[k * kTS + tid] = acc * gelu_grad(z1);
        }
        __syncthreads();
        // dW1 = d1^T x, db1 = sum d1
        if (tid < kMlpH) {
            float a0 = 0.f, a1 = 0.f, b = 0.f;
            for (int s = 0; s < kTrainThreads; ++s) {
                const float d = S.q[tid * kTS + s];
                a0 = fmaf(d, S.x[0][s], a0);
                a1 = fmaf(d, S.x[1][s], a1);
                b += d;
            }
            S.g[kOffW1 + 2 * tid] += a0;
            S.g[kOffW1 + 2 * tid + 1] += a1;
            S.g[kOffB1 + tid] += b;
        }
        __syncthreads();
    }
    S.dy[tid] = my_loss;  // (the per-sample buffer is free after the last pass)
    __syncthreads();
    float *slot = part + (size_t)blockIdx.x * (kMlpParams + 1);
    for (int i = tid; i < kMlpParams; i += blockDim.x) slot[i] = S.g[i];
    if (tid == 0) {
        float l = 0.f;
        for (int s = 0; s < kTrainThreads; ++s) l += S.dy[s];
        slot[kMlpParams] = l * inv_n;
    }
}

// the training kernel's per-CTA slots summed in CTA order: the gradient, and
// the batch's mean loss into loss_out
__global__ void mlp_reduce_kernel(const float *__restrict__ part, int slots, float *grad, float *loss_out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > kMlpParams) return;
    float a = 0.f;
    for (int c = 0; c < slots; ++c) a += part[(size_t)c * (kMlpParams + 1) + i];
    if (i < kMlpParams)
        grad[i] = a;
    else
        *loss_out = a;
}

// Adam (Kingma & Ba 2015); refreshes the bf16 copy and clears the gradient
__global__ void mlp_adam_kernel(float *p, float *m, float *v, float *g, __nv_bfloat16 *w, float lr, float bc1,
                                float bc2)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kMlpParams; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = 0.9f * m[i] + 0.1f * gi;
        const float vi = 0.999f * v[i] + 0.001f * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + 1e-8f);
        p[i] = pi;
        w[i] = __float2bfloat16_rn(pi);
        g[i] = 0.f;
    }
}

// ---------------------------------------------------------------------------
// batch inference on the fifth-generation tensor cores.  One CTA of 1024
// threads per SM, eight independent groups of 128 (four warps each); a group
// takes a tile of 128 samples per pass, thread t owning sample t (row t of the
// group's A operand, lane t of its tensor-memory accumulator).  Each CTA owns
// an equal contiguous range of tiles, and its groups claim the tiles of that
// range one at a time from a shared-memory counter: the warp schedulers favour
// some warps over others, and with a fixed share per group the favoured groups
// finished early and left their SM short of warps for the rest of the launch
// (a quarter of the warp slots idle on average).  Per tile:
//   1. thread t writes its features into columns 64..79 of row t: x1 and x2
//      each as three bf16 parts (h + m + l = x exactly: a float's 24 bits in
//      three pieces of 8), a 1 and zeros;
//   2. one thread issues layer 1 as one M = 128, N = 64, K = 16 MMA of those
//      columns against [w1a w1a w1a w1b w1b w1b b1 0 ...] (the bias rides on
//      the 1), commits it to the group's mbarrier;
//   3. every thread reads its row's 64 FP32 sums back (tcgen05.ld), applies
//      2 gelu and writes them, rounded to bf16, into columns 0..63 of its row;
//   4. one thread issues layer 2 as five K = 16 MMAs: columns 0..63 against
//      W2 / 2, then columns 64..79 against [0 0 0 0 0 0 b2 0 ...], which adds
//      b2 through the same 1 (the accumulator of step 2 is overwritten);
//   5. every thread reads its 64 sums back for bias-free GELU and layer 3
//      (W3 / 2 and b3 on the CUDA cores).
// Products of bf16 values are exact in the FP32 accumulator, so layer 1 is the
// FP32 sum w1a x1 + w1b x2 + b1 up to the accumulation order.  The groups
// synchronise only among themselves (named barriers), so one group's GELUs
// overlap the other's MMAs.  (The event kernels evaluate the network 32
// samples per warp inside their own loops and keep the warp-level mma.sync
// form of mlp_forward_warp.)
// ---------------------------------------------------------------------------
constexpr int kTcGroups = 8;
constexpr int kTcTile = 128;
constexpr int kTcThreads = kTcGroups * kTcTile;  // 1024
constexpr int kTcK = kMlpH + 16;                 // the A operand's columns: activations, then features
constexpr uint32_t kTcCols = kTcGroups * kMlpH;  // one FP32 accumulator of N = 64 columns per group: all 512

struct TcSmem {
    __nv_bfloat16 a[kTcGroups][kTcTile * kTcK];  // each group's A operand [m][k] (K-major, K = 80)
    __nv_bfloat16 b2[kMlpH * kTcK];              // [W2 / 2 | b2 column] [n][k] (K-major, K = 80)
    __nv_bfloat16 b1[kMlpH * 16];                // layer 1 against the split features [n][k] (K = 16)
    alignas(16) float w3[kMlpH];                 // W3 / 2
    float b3;
    alignas(8) uint64_t bar[kTcGroups];
    uint32_t tmem;
    int fail[kTcGroups];
    int next;                                    // tiles of the CTA's range handed out so far
    int claim[kTcGroups];                        // each group's tile two passes ahead
};
// One CTA per SM (its registers and shared memory leave room for no second
// one), holding all 512 TMEM columns, so no TMEM allocation waits.
constexpr int kTcSmemBytes = (int)((sizeof(TcSmem) + 127) / 128 * 128);
static_assert(kTcSmemBytes + 1024 <= 228 * 1024 && 2 * (kTcSmemBytes + 1024) > 228 * 1024,
              "shared memory of the tensor-core sampler must admit exactly one CTA per SM");

__device__ __forceinline__ void group_sync(int group)
{
    asm volatile("bar.sync %0, %1;" ::"r"(1 + group), "r"(kTcTile) : "memory");
}

__device__ __forceinline__ uint16_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }

// x = h + m + l exactly, each a bf16 (round to nearest at every cut: the
// remainders x - h and x - h - m are exact in FP32 and have at most 16 and 8
// significant bits)
__device__ __forceinline__ void split3(float x, uint16_t &h, uint16_t &m, uint16_t &l)
{
    h = bf16_bits(x);
    const float r1 = x - __uint_as_float((uint32_t)h << 16);
    m = bf16_bits(r1);
    const float r2 = r1 - __uint_as_float((uint32_t)m << 16);
    l = bf16_bits(r2);
}

__device__ __forceinline__ uint32_t pack16(uint16_t lo, uint16_t hi) { return (uint32_t)lo | ((uint32_t)hi << 16); }

// columns 64..71 of a sample's A row: x1 and x2 in three bf16 parts each, 1, 0
__device__ __forceinline__ uint4 feature_row(const MlpIn &in)
{
    uint16_t h1, m1, l1, h2, m2, l2;
    split3(in.x1, h1, m1, l1);
    split3(in.x2, h2, m2, l2);
    return make_uint4(pack16(h1, m1), pack16(l1, h2), pack16(m2, l2), pack16(0x3f80u, 0));
}

__global__ void __launch_bounds__(kTcThreads, 1) mlp_sample_tc_kernel(MlpView v, const double *__restrict__ chi,
                                                                     const double *__restrict__ uu, int64_t n,
                                                                     double *__restrict__ xi)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TcSmem &S = *reinterpret_cast<TcSmem *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, grp = tid / kTcTile, row = tid % kTcTile;
    unsigned char *const b2raw = reinterpret_cast<unsigned char *>(S.b2);
    // W2 is staged halved (exact): the activations are 2 gelu (gelu2x)
    for (int i = tid; i < kMlpH * kMlpH; i += kTcThreads)
        *reinterpret_cast<__nv_bfloat16 *>(b2raw + core_offset<kTcK>(i / kMlpH, i % kMlpH)) =
            __float2bfloat16_rn(0.5f * __bfloat162float(v.w[kOffW2 + i]));
    if (tid < kMlpH) {
        const int r = tid;
        const uint16_t wa = __bfloat16_as_ushort(v.w[kOffW1 + 2 * r]), wb = __bfloat16_as_ushort(v.w[kOffW1 + 2 * r + 1]);
        const uint16_t c1 = __bfloat16_as_ushort(v.w[kOffB1 + r]), c2 = __bfloat16_as_ushort(v.w[kOffB2 + r]);
        unsigned char *b1raw = reinterpret_cast<unsigned char *>(S.b1);
        // layer 1 row r: the weights of x1's and x2's three parts, b1 on the 1
        *reinterpret_cast<uint4 *>(b1raw + core_offset<16>(r, 0)) =
            make_uint4(pack16(wa, wa), pack16(wa, wb), pack16(wb, wb), pack16(c1, 0));
        *reinterpret_cast<uint4 *>(b1raw + core_offset<16>(r, 8)) = make_uint4(0, 0, 0, 0);
        // layer 2 row r, columns 64..79: b2 on the 1, zero against the features
        *reinterpret_cast<uint4 *>(b2raw + core_offset<kTcK>(r, kMlpH)) = make_uint4(0, 0, 0, pack16(c2, 0));
        *reinterpret_cast<uint4 *>(b2raw + core_offset<kTcK>(r, kMlpH + 8)) = make_uint4(0, 0, 0, 0);
        S.w3[r] = 0.5f * __bfloat162float(v.w[kOffW3 + r]);
    }
    unsigned char *const arow = reinterpret_cast<unsigned char *>(S.a[grp]) + core_offset<kTcK>(row, 0);
    *reinterpret_cast<uint4 *>(arow + core_offset<kTcK>(0, kMlpH + 8)) = make_uint4(0, 0, 0, 0);  // never rewritten
    if (tid == 0) {
        S.b3 = __bfloat162float(v.w[kOffB3]);
        for (int g = 0; g < kTcGroups; ++g) {
            S.fail[g] = 0;
            mbar_init(&S.bar[g], 1);
        }
        S.next = 2 * kTcGroups;  // the first two tiles of every group are fixed (below)
        mbar_fence_init();
    }
    if (warp == 0) tmem_alloc(&S.tmem, kTcCols);
    fence_async_smem();  // the operands were written by ordinary stores and are read by the tensor core
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = S.tmem;
    constexpr uint32_t idesc = idesc_bf16_f32(kTcTile, kMlpH);
    // (the operand descriptors are formed where the issuing thread needs them,
    // which keeps them out of the other threads' registers)
    constexpr uint64_t kFeat = (uint64_t)(kMlpH / 8 * 128 >> 4);  // descriptor step to columns 64..79
    const uint32_t dacc = tmem + (uint32_t)(grp * kMlpH);          // the group's accumulator (lane 0)
    // this thread's row: TMEM lane 32 (warp % 4) + lane
    const uint32_t tacc = dacc + ((uint32_t)((warp & 3) * 32) << 16);
    uint32_t parity = 0;
    // the CTA's tiles t_begin + [0, t_len); group g starts on its tiles g and
    // g + kTcGroups, then claims one tile per pass from S.next (tile numbers
    // relative to t_begin: a CTA's range stays far below 2^31 tiles)
    const int64_t n_tiles = (n + kTcTile - 1) / kTcTile;
    const int64_t t_begin = (int64_t)blockIdx.x * n_tiles / gridDim.x;
    const int t_len = (int)(((int64_t)blockIdx.x + 1) * n_tiles / gridDim.x - t_begin);
    const int64_t s_begin = t_begin * kTcTile + row;  // this thread's sample in tile 0
    int t_cur = grp, t_nxt = grp + kTcGroups;
    // Software pipeline within the group: the features of tile k + 1 are formed
    // while the layer-2 MMAs of tile k run, the output map of tile k while the
    // layer-1 MMA of tile k + 1 runs, and (chi, U) are loaded two tiles ahead.
    const int64_t i0 = s_begin + (int64_t)t_cur * kTcTile, i1 = s_begin + (int64_t)t_nxt * kTcTile;
    const bool v0 = t_cur < t_len && i0 < n, v1 = t_nxt < t_len && i1 < n;
    MlpIn in = mlp_input(v, v0 ? chi[i0] : 1.0, v0 ? uu[i0] : 0.5);
    uint4 feat = feature_row(in);
    double c_next = v1 ? chi[i1] : 1.0;
    double u_next = v1 ? uu[i1] : 0.5;
    MlpIn in_prev = in;
    int64_t i_prev = n;  // (no previous tile yet)
    float y_prev = 0.0f;
    // A wait that gives up (never expected) sets the group's flag; from the
    // next barrier on, the group issues no MMA, waits for none and writes NaN,
    // but keeps passing the same barriers, so that no thread waits for one that
    // left the loop.
    while (t_cur < t_len) {
        const int64_t i = s_begin + (int64_t)t_cur * kTcTile;
        *reinterpret_cast<uint4 *>(arow + core_offset<kTcK>(0, kMlpH)) = feat;
        if (row == 0) S.claim[grp] = atomicAdd(&S.next, 1);  // (read by the group after the barrier)
        fence_async_smem();
        tc_fence_before();  // (orders the previous tile's accumulator loads before the barrier)
        group_sync(grp);
        const int t_nn = S.claim[grp];  // (rewritten only after the group's next barrier)
        bool live = S.fail[grp] == 0;
        if (live && row == 0) {
            tc_fence_after();
            const uint64_t adesc = smem_desc(smem_u32(S.a[grp]), 128, kTcK * 16);
            tc_mma_bf16(dacc, adesc + kFeat, smem_desc(smem_u32(S.b1), 128, 16 * 16), idesc, false);  // layer 1
            tc_commit(&S.bar[grp]);
        }
        if (i_prev < n) xi[i_prev] = mlp_output(v.proc, y_prev, in_prev);  // the previous tile (NaN y: NaN)
        bool ok = live && mbar_wait(&S.bar[grp], parity);
        if (live) parity ^= 1u;
        if (live && !ok) {
            S.fail[grp] = 1;  // seen by the whole group after its next barrier
            note_error(QED_EW_WAIT_TIMEOUT);
        }
        if (ok) {
            tc_fence_after();
#pragma unroll
            for (int c0 = 0; c0 < kMlpH; c0 += 16) {
                uint32_t ra[16];
                tc_ld16(tacc + (uint32_t)c0, ra);
                tc_wait_ld();
#pragma unroll
                for (int kc = 0; kc < 2; ++kc) {  // eight columns, one 16-byte store
                    uint32_t w[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int e = 8 * kc + 2 * q;
                        const uint32_t r0 = ra[e], r1 = ra[e + 1];
                        const float2 g = f2u(gelu2x(f2(__uint_as_float(r0), __uint_as_float(r1))));
                        w[q] = pack_bf16(g.x, g.y);
                    }
                    *reinterpret_cast<uint4 *>(arow + core_offset<kTcK>(0, c0 + 8 * kc)) =
                        make_uint4(w[0], w[1], w[2], w[3]);
                }
            }
        }
        fence_async_smem();
        tc_fence_before();  // (the layer-1 loads complete before layer 2 overwrites the accumulator)
        group_sync(grp);
        live = S.fail[grp] == 0;
        if (live && row == 0) {
            tc_fence_after();
            // layer 2: Z = H1 W2^T / 2 + b2, K = 80 in five steps of 16 (two core matrices, 256 bytes)
            const uint64_t adesc = smem_desc(smem_u32(S.a[grp]), 128, kTcK * 16);
            const uint64_t b2desc = smem_desc(smem_u32(S.b2), 128, kTcK * 16);
#pragma unroll
            for (int kk = 0; kk < kTcK / 16; ++kk) {
                const uint64_t step = (uint64_t)(kk * 256 >> 4);
                tc_mma_bf16(dacc, adesc + step, b2desc + step, idesc, kk > 0);
            }
            tc_commit(&S.bar[grp]);
        }
        in_prev = in;
        i_prev = i;
        in = mlp_input(v, c_next, u_next);
        feat = feature_row(in);
        const int64_t j = s_begin + (int64_t)t_nn * kTcTile;
        const bool vj = t_nn < t_len && j < n;
        c_next = vj ? chi[j] : 1.0;
        u_next = vj ? uu[j] : 0.5;
        t_cur = t_nxt;
        t_nxt = t_nn;
        ok = live && mbar_wait(&S.bar[grp], parity);
        if (live) parity ^= 1u;
        if (live && !ok) {
            S.fail[grp] = 1;
            note_error(QED_EW_WAIT_TIMEOUT);
        }
        float y = __int_as_float(0x7fc00000);
        if (ok) {
            tc_fence_after();
            // GELU and layer 3 on this thread's 64 accumulators, in pairs
            uint64_t y2 = f2(S.b3, 0.0f);
#pragma unroll
            for (int c0 = 0; c0 < kMlpH; c0 += 16) {
                uint32_t ra[16];
                tc_ld16(tacc + (uint32_t)c0, ra);
                tc_wait_ld();
#pragma unroll
                for (int q = 0; q < 16; q += 4) {
                    const ulonglong2 w3 = *reinterpret_cast<const ulonglong2 *>(S.w3 + c0 + q);
                    y2 = ffma2(w3.x, gelu2x(f2(__uint_as_float(ra[q]), __uint_as_float(ra[q + 1]))), y2);
                    y2 = ffma2(w3.y, gelu2x(f2(__uint_as_float(ra[q + 2]), __uint_as_float(ra[q + 3]))), y2);
                }
            }
            const float2 yy = f2u(y2);
            y = yy.x + yy.y;
        }
        y_prev = y;
    }
    if (i_prev < n) xi[i_prev] = mlp_output(v.proc, y_prev, in_prev);
    tc_fence_before();
    __syncthreads();
    if (S.fail[grp]) mbar_wait(&S.bar[grp], parity ^ 1u);  // one more bounded wait for an MMA in flight
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_free(tmem, kTcCols);
    }
}

// batch inverse-CDF sampling through the 2-D tables (the path the network replaces)
template <typename T>
__global__ void table_sample_kernel(Table2D<T> tb, int proc, const double *__restrict__ chi,
                                    const double *__restrict__ uu, int64_t n, double *__restrict__ xi)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double u = uu[i];
        if (proc == QED_PROC_QS) {
            xi[i] = (double)qs_sample_xi<T>(tb, (T)chi[i], sample_uniform<T>(u));
        } else {
            bool electron;
            const T xs = bw_sample_xi<T>(tb, (T)chi[i], u, electron);
            xi[i] = electron ? (double)xs : 1.0 - (double)xs;
        }
    }
}

static qed_status check_mlp(const qed_mlp *m, int proc)
{
    if (!m) QED_FAIL(QED_ERR_INVALID_ARG, "mlp handle is NULL");
    if (proc != QED_PROC_QS && proc != QED_PROC_BW) QED_FAIL(QED_ERR_INVALID_ARG, "bad process %d", proc);
    return QED_OK;
}

size_t infer_smem_bytes() { return sizeof(InferSmem); }

}  // namespace qed

using namespace qed;

static void free_mlp(qed_mlp *m)
{
    if (!m) return;
    for (int p = 0; p < 2; ++p) {
        void *ptrs[] = {m->master[p], m->adam_m[p], m->adam_v[p], m->grad[p], m->part[p], m->loss[p], m->w[p]};
        for (void *x : ptrs)
            if (x) cudaFree(x);
    }
    delete m;
}

// both networks for the given chi ranges (index: process), weights from Philox(seed)
static qed_status create_mlp(const double chi_min[2], const double chi_max[2], uint64_t seed, qed_mlp **out,
                             cudaStream_t st)
{
    qed_mlp *m = new qed_mlp();
    memset(m, 0, sizeof(*m));
    cudaGetDevice(&m->device);
    for (int p = 0; p < 2; ++p) m->chi_min[p] = chi_min[p], m->chi_max[p] = chi_max[p];
    m->part_slots = sm_count();
    for (int p = 0; p < 2; ++p) {
        cudaError_t e = cudaSuccess;
        float **fp[] = {&m->master[p], &m->adam_m[p], &m->adam_v[p], &m->grad[p]};
        for (float **f : fp)
            if (e == cudaSuccess) e = cudaMalloc((void **)f, kMlpParams * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc((void **)&m->loss[p], sizeof(float));
        if (e == cudaSuccess)
            e = cudaMalloc((void **)&m->part[p], (size_t)m->part_slots * (kMlpParams + 1) * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc((void **)&m->w[p], kMlpParams * sizeof(__nv_bfloat16));
        if (e == cudaSuccess) e = cudaMemsetAsync(m->adam_m[p], 0, kMlpParams * sizeof(float), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(m->adam_v[p], 0, kMlpParams * sizeof(float), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(m->grad[p], 0, kMlpParams * sizeof(float), st);
        if (e == cudaSuccess) e = cudaMemsetAsync(m->loss[p], 0, sizeof(float), st);
        if (e != cudaSuccess) {
            free_mlp(m);
            QED_FAIL(QED_ERR_CUDA, "mlp allocation failed: %s", cudaGetErrorString(e));
        }
        mlp_init_kernel<<<(kMlpParams + 255) / 256, 256, 0, st>>>(m->master[p], seed, p);
        mlp_to_bf16_kernel<<<(kMlpParams + 255) / 256, 256, 0, st>>>(m->master[p], m->w[p]);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        free_mlp(m);
        QED_FAIL(QED_ERR_CUDA, "mlp initialisation failed: %s", cudaGetErrorString(e));
    }
    *out = m;
    return QED_OK;
}

extern "C" qed_status qed_mlp_create(const qed_tables *t, uint64_t seed, qed_mlp **out, void *stream)
{
    clear_error();
    qed_status s;
    if (!out) QED_FAIL(QED_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if ((s = check_tables(t))) return s;
    const double lo[2] = {t->params.qs.chi_min, t->params.bw.chi_min};
    const double hi[2] = {t->params.qs.chi_max, t->params.bw.chi_max};
    return create_mlp(lo, hi, seed, out, as_stream(stream));
}

// ---------------------------------------------------------------------------
// file format: "QEDMLP\0\1" | u32 version | u32 parameters per network |
// chi_min[2] | chi_max[2] (FP64) | QS then BW FP32 master parameters
// (little-endian host order) | u64 FNV-1a of everything before it
// ---------------------------------------------------------------------------
static const char kMlpMagic[8] = {'Q', 'E', 'D', 'M', 'L', 'P', 0, 1};
static const uint32_t kMlpFileVersion = 1;
static const size_t kMlpFileHead = 8 + 4 + 4 + 4 * 8;
static const size_t kMlpFileBody = 2 * (size_t)kMlpParams * sizeof(float);

extern "C" qed_status qed_mlp_save(const qed_mlp *m, const char *path)
{
    clear_error();
    qed_status s = check_mlp(m, QED_PROC_QS);
    if (s) return s;
    if (!path) QED_FAIL(QED_ERR_INVALID_ARG, "path is NULL");
    std::vector<unsigned char> buf(kMlpFileHead + kMlpFileBody);
    unsigned char *q = buf.data();
    const uint32_t n_params = kMlpParams;
    memcpy(q, kMlpMagic, 8);
    memcpy(q + 8, &kMlpFileVersion, 4);
    memcpy(q + 12, &n_params, 4);
    memcpy(q + 16, m->chi_min, 16);
    memcpy(q + 32, m->chi_max, 16);
    for (int p = 0; p < 2; ++p)
        if ((s = qed_mlp_get_params(m, (qed_process)p, (float *)(q + kMlpFileHead) + (size_t)p * kMlpParams)))
            return s;
    const uint64_t h = fnv1a64(buf.data(), buf.size());
    FILE *f = fopen(path, "wb");
    if (!f) QED_FAIL(QED_ERR_IO, "cannot open %s for writing", path);
    bool ok = fwrite(buf.data(), 1, buf.size(), f) == buf.size() && fwrite(&h, 8, 1, f) == 1;
    ok = (fclose(f) == 0) && ok;
    if (!ok) QED_FAIL(QED_ERR_IO, "write to %s failed", path);
    return QED_OK;
}

extern "C" qed_status qed_mlp_load(const char *path, qed_mlp **out, void *stream)
{
    clear_error();
    if (!path || !out) QED_FAIL(QED_ERR_INVALID_ARG, "path/out is NULL");
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f) QED_FAIL(QED_ERR_IO, "cannot open %s", path);
    std::vector<unsigned char> buf(kMlpFileHead + kMlpFileBody + 8 + 1);
    const size_t got = fread(buf.data(), 1, buf.size(), f);
    fclose(f);
    if (got != kMlpFileHead + kMlpFileBody + 8) QED_FAIL(QED_ERR_IO, "%s: size %zu, not a network file", path, got);
    if (memcmp(buf.data(), kMlpMagic, 8) != 0) QED_FAIL(QED_ERR_IO, "%s: bad magic", path);
    uint32_t ver, n_params;
    memcpy(&ver, buf.data() + 8, 4);
    memcpy(&n_params, buf.data() + 12, 4);
    if (ver != kMlpFileVersion) QED_FAIL(QED_ERR_IO, "%s: unsupported version %u", path, ver);
    if (n_params != (uint32_t)kMlpParams) QED_FAIL(QED_ERR_IO, "%s: %u parameters per network, not %d", path, n_params, kMlpParams);
    uint64_t h;
    memcpy(&h, buf.data() + kMlpFileHead + kMlpFileBody, 8);
    if (h != fnv1a64(buf.data(), kMlpFileHead + kMlpFileBody)) QED_FAIL(QED_ERR_IO, "%s: checksum mismatch", path);
    double lo[2], hi[2];
    memcpy(lo, buf.data() + 16, 16);
    memcpy(hi, buf.data() + 32, 16);
    for (int p = 0; p < 2; ++p)
        if (!(lo[p] > 0 && hi[p] > lo[p] && std::isfinite(hi[p])))
            QED_FAIL(QED_ERR_IO, "%s: bad chi range [%g, %g]", path, lo[p], hi[p]);
    std::vector<float> params(2 * (size_t)kMlpParams);
    memcpy(params.data(), buf.data() + kMlpFileHead, kMlpFileBody);
    for (float v : params)
        if (!std::isfinite(v)) QED_FAIL(QED_ERR_IO, "%s: non-finite parameter", path);
    qed_mlp *m = nullptr;
    qed_status s = create_mlp(lo, hi, 0, &m, as_stream(stream));
    if (s) return s;
    for (int p = 0; p < 2; ++p)
        if ((s = qed_mlp_set_params(m, (qed_process)p, params.data() + (size_t)p * kMlpParams, stream))) {
            free_mlp(m);
            return s;
        }
    *out = m;
    return QED_OK;
}

extern "C" qed_status qed_mlp_destroy(qed_mlp *m)
{
    clear_error();
    free_mlp(m);
    return QED_OK;
}

extern "C" qed_status qed_mlp_get_params(const qed_mlp *m, qed_process proc, float *host_params)
{
    clear_error();
    qed_status s = check_mlp(m, proc);
    if (s) return s;
    if (!host_params) QED_FAIL(QED_ERR_INVALID_ARG, "host_params is NULL");
    QED_CUDA_TRY(cudaMemcpy(host_params, m->master[proc], kMlpParams * sizeof(float), cudaMemcpyDeviceToHost));
    return QED_OK;
}

extern "C" qed_status qed_mlp_set_params(qed_mlp *m, qed_process proc, const float *host_params, void *stream)
{
    clear_error();
    qed_status s = check_mlp(m, proc);
    if (s) return s;
    if (!host_params) QED_FAIL(QED_ERR_INVALID_ARG, "host_params is NULL");
    cudaStream_t st = as_stream(stream);
    QED_CUDA_TRY(cudaMemcpyAsync(m->master[proc], host_params, kMlpParams * sizeof(float), cudaMemcpyHostToDevice, st));
    mlp_to_bf16_kernel<<<(kMlpParams + 255) / 256, 256, 0, st>>>(m->master[proc], m->w[proc]);
    QED_LAUNCH_CHECK();
    QED_CUDA_TRY(cudaMemsetAsync(m->adam_m[proc], 0, kMlpParams * sizeof(float), st));
    QED_CUDA_TRY(cudaMemsetAsync(m->adam_v[proc], 0, kMlpParams * sizeof(float), st));
    QED_CUDA_TRY(cudaStreamSynchronize(st));
    m->step[proc] = 0;
    return QED_OK;
}

static qed_status launch_train(qed_mlp *m, int proc, const double *chi, const double *u, const double *xi, int64_t n,
                               cudaStream_t st)
{
    static bool attr = false;
    const size_t sm = sizeof(TrainSmem);
    if (!attr) {
        QED_CUDA_TRY(cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        attr = true;
    }
    int64_t blocks = (n + kTrainThreads - 1) / kTrainThreads;
    const int64_t cap = (int64_t)m->part_slots;
    blocks = blocks < 1 ? 1 : (blocks > cap ? cap : blocks);
    mlp_train_kernel<<<(int)blocks, kTrainThreads, sm, st>>>(mlp_view(m, proc), chi, u, xi, n, m->part[proc]);
    QED_LAUNCH_CHECK();
    mlp_reduce_kernel<<<(kMlpParams + 1 + 255) / 256, 256, 0, st>>>(m->part[proc], (int)blocks, m->grad[proc],
                                                                   m->loss[proc]);
    QED_LAUNCH_CHECK();
    return QED_OK;
}

// training needs samples (empty = 0 allowed only where nothing is computed from them)
static qed_status check_batch(const double *chi, const double *u, const double *xi, int64_t n, bool empty_ok = false)
{
    if (n < 0 || (n == 0 && !empty_ok)) QED_FAIL(QED_ERR_INVALID_ARG, "batch size must be positive");
    if (n > 0 && (!chi || !u || !xi)) QED_FAIL(QED_ERR_INVALID_ARG, "a batch array is NULL");
    return QED_OK;
}

extern "C" qed_status qed_mlp_gradients(qed_mlp *m, qed_process proc, const double *d_chi, const double *d_u,
                                        const double *d_xi, int64_t n, float *d_grad, float *d_loss, void *stream)
{
    clear_error();
    qed_status s;
    if ((s = check_mlp(m, proc))) return s;
    if ((s = check_batch(d_chi, d_u, d_xi, n))) return s;
    if (!d_grad) QED_FAIL(QED_ERR_INVALID_ARG, "d_grad is NULL");
    cudaStream_t st = as_stream(stream);
    QED_CUDA_TRY(cudaMemsetAsync(m->grad[proc], 0, kMlpParams * sizeof(float), st));
    if ((s = launch_train(m, proc, d_chi, d_u, d_xi, n, st))) return s;
    QED_CUDA_TRY(cudaMemcpyAsync(d_grad, m->grad[proc], kMlpParams * sizeof(float), cudaMemcpyDeviceToDevice, st));
    if (d_loss) QED_CUDA_TRY(cudaMemcpyAsync(d_loss, m->loss[proc], sizeof(float), cudaMemcpyDeviceToDevice, st));
    QED_CUDA_TRY(cudaMemsetAsync(m->grad[proc], 0, kMlpParams * sizeof(float), st));
    return QED_OK;
}

extern "C" qed_status qed_mlp_train_step(qed_mlp *m, qed_process proc, const double *d_chi, const double *d_u,
                                         const double *d_xi, int64_t n, float lr, float *d_loss, void *stream)
{
    clear_error();
    qed_status s;
    if ((s = check_mlp(m, proc))) return s;
    if ((s = check_batch(d_chi, d_u, d_xi, n))) return s;
    if (!(lr > 0.f)) QED_FAIL(QED_ERR_INVALID_ARG, "learning rate must be positive");
    cudaStream_t st = as_stream(stream);
    if ((s = launch_train(m, proc, d_chi, d_u, d_xi, n, st))) return s;
    const int64_t k = ++m->step[proc];
    const float bc1 = 1.f - powf(0.9f, (float)k), bc2 = 1.f - powf(0.999f, (float)k);
    mlp_adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, st>>>(m->master[proc], m->adam_m[proc], m->adam_v[proc],
                                                              m->grad[proc], m->w[proc], lr, bc1, bc2);
    QED_LAUNCH_CHECK();
    if (d_loss) QED_CUDA_TRY(cudaMemcpyAsync(d_loss, m->loss[proc], sizeof(float), cudaMemcpyDeviceToDevice, st));
    return QED_OK;
}

extern "C" qed_status qed_mlp_sample(const qed_mlp *m, qed_process proc, const double *d_chi, const double *d_u,
                                     int64_t n, double *d_xi, void *stream)
{
    clear_error();
    qed_status s;
    if ((s = check_mlp(m, proc))) return s;
    if ((s = check_batch(d_chi, d_u, d_xi, n, true))) return s;
    if (n == 0) return QED_OK;
    static bool attr = false;
    if (!attr) {
        // the largest shared-memory carveout (the CTA takes 177 KB)
        QED_CUDA_TRY(
            cudaFuncSetAttribute(mlp_sample_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemBytes));
        QED_CUDA_TRY(cudaFuncSetAttribute(mlp_sample_tc_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                          (int)cudaSharedmemCarveoutMaxShared));
        attr = true;
    }
    // one CTA per SM (it holds all of the SM's TMEM), fewer for small batches
    const int64_t want = (n + (int64_t)kTcGroups * kTcTile - 1) / ((int64_t)kTcGroups * kTcTile),
                  cap = (int64_t)sm_count();
    const int blocks = (int)(want < cap ? want : cap);
    mlp_sample_tc_kernel<<<blocks, kTcThreads, kTcSmemBytes, as_stream(stream)>>>(mlp_view(m, proc), d_chi, d_u, n,
                                                                                 d_xi);
    QED_LAUNCH_CHECK();
    return QED_OK;
}

extern "C" qed_status qed_table_sample(const qed_tables *t, qed_process proc, qed_precision prec, const double *d_chi,
                                       const double *d_u, int64_t n, double *d_xi, void *stream)
{
    clear_error();
    qed_status s;
    if ((s = check_tables(t))) return s;
    if (proc != QED_PROC_QS && proc != QED_PROC_BW) QED_FAIL(QED_ERR_INVALID_ARG, "bad process %d", (int)proc);
    if ((s = check_batch(d_chi, d_u, d_xi, n, true))) return s;
    if (n == 0) return QED_OK;
    cudaStream_t st = as_stream(stream);
    if (prec == QED_F32) {
        TablesView<float> v = make_view<float>(t);
        const int g = resident_grid<table_sample_kernel<float>>(256, 0, n);
        table_sample_kernel<float><<<g, 256, 0, st>>>(proc == QED_PROC_QS ? v.qs_P : v.bw_P, proc, d_chi, d_u, n,
                                                      d_xi);
    } else {
        TablesView<double> v = make_view<double>(t);
        const int g = resident_grid<table_sample_kernel<double>>(256, 0, n);
        table_sample_kernel<double><<<g, 256, 0, st>>>(proc == QED_PROC_QS ? v.qs_P : v.bw_P, proc, d_chi, d_u, n,
                                                       d_xi);
    }
    QED_LAUNCH_CHECK();
    return QED_OK;
}
