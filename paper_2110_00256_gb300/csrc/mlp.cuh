// mlp.cuh -- the learned inverse-CDF sampler: a 2-64-64-1 GELU network per
// process, bfloat16 weights, FP32 accumulation, the 64x64 layer on the tensor
// cores.  The paper has no learned sampler: this stands in for the 2-D
// inverse-CDF tables of §3.1 and §3.2.
//
// Inputs (chi, U) -> features x1 = ln chi_c scaled to [-1, 1] over the chi
// range (chi_c = chi clamped into it), x2 = 2 U - 1 (QS) or 4 min(U, 1 - U) - 1
// (BW).  Output maps (centred and scaled so that the network's output y is of
// order one over the whole chi range):
//   QS: ln(xi / (1 - xi)) = y + 3 ln U + L(chi_c),  L(chi) = ln(chi / (1 + chi))
//       (xi ~ U^3 as U -> 0, xi scales with chi for small chi, and the logit
//       resolves the hard end xi -> 1 in 1 - xi);
//   BW: the folded fraction of the lepton U selects (U <= 1/2: the electron)
//       xi_s = min(1/2, 1 / (1 + exp(4 w(chi_c) y))),  w(chi) = sqrt(chi / (chi + 16/3)) / 2
//       (for small chi the pair split concentrates around 1/2 with a width
//       ~ sqrt(3 chi / 64), where the map is 1/2 - w y to first order; for large
//       chi the folded split crowds towards 0, which the logit resolves).
// Activation: GELU in its tanh form, the FP32 arithmetic in packed pairs
// (f32x2) and tanh.approx.f32 (~2^-11), the same instructions in training and
// in every inference path.
//
// Parameter vector (kMlpParams floats, bf16 on the device for inference):
// W1[64][2], b1[64], W2[64][64], b2[64], W3[64], b3.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace qed {

constexpr int kMlpH = 64;
constexpr int kMlpParams = kMlpH * 2 + kMlpH + kMlpH * kMlpH + kMlpH + kMlpH + 1;  // 4417
constexpr int kOffW1 = 0, kOffB1 = 128, kOffW2 = 192, kOffB2 = 192 + 4096, kOffW3 = kOffB2 + 64, kOffB3 = kOffW3 + 64;
constexpr int kMlpPad = 72;  // bf16 row stride of the shared 64-wide tiles (conflict-free fragment loads)

// input normalisation of one process: x1 = (ln chi_c - ln_min) * scale - 1
struct MlpView {
    const __nv_bfloat16 *w;  // kMlpParams bf16
    float ln_min, ln_max, scale;
    int proc;                // QED_PROC_QS or QED_PROC_BW
};

__device__ __forceinline__ float tanh_approx(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// ---- packed FP32 pairs (two lanes of one 64-bit register) ------------------
__device__ __forceinline__ uint64_t f2(float lo, float hi)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float2 f2u(uint64_t r)
{
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
__device__ __forceinline__ uint64_t ffma2(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ uint64_t fmul2(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ uint64_t fadd2(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// tanh of both lanes (tanh.approx.f32, |relative error| < 2^-10.99).  Measured
// against tanh.approx.f16x2 on the pair: one special-function operation fewer per
// pair, but the conversions to and from FP16 cost more issue slots than that saves
// (the sampler ran 12 % faster with this form)
__device__ __forceinline__ uint64_t tanh2(uint64_t u)
{
    const float2 v = f2u(u);
    return f2(tanh_approx(v.x), tanh_approx(v.y));
}

// gelu(x) = x/2 (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3)))  (Hendrycks & Gimpel)
// on both lanes: h = x/2, u = x (sqrt(2/pi) + sqrt(2/pi) 0.044715 x^2), h + h tanh(u)
// (FP32 pairs; the same speed as the whole GELU on FP16 pairs, measured, and more precise)
__device__ __forceinline__ uint64_t gelu2(uint64_t x)
{
    const uint64_t c1 = f2(0.035677408136300125f, 0.035677408136300125f);
    const uint64_t c0 = f2(0.7978845608028654f, 0.7978845608028654f);
    const uint64_t half = f2(0.5f, 0.5f);
    const uint64_t u = fmul2(x, ffma2(c1, fmul2(x, x), c0));
    const uint64_t h = fmul2(half, x);
    return ffma2(h, tanh2(u), h);
}

// 2 gelu(x) = x + x tanh(u) on both lanes, bit for bit twice gelu2 (halving is
// exact in binary floating point): the tensor-core sampler folds the 1/2 into the
// next layer's weights (W2 / 2, W3 / 2, also exact), one multiply less per GELU
__device__ __forceinline__ uint64_t gelu2x(uint64_t x)
{
    const uint64_t c1 = f2(0.035677408136300125f, 0.035677408136300125f);
    const uint64_t c0 = f2(0.7978845608028654f, 0.7978845608028654f);
    const uint64_t u = fmul2(x, ffma2(c1, fmul2(x, x), c0));
    return ffma2(x, tanh2(u), x);
}

// one lane of gelu2 (the same arithmetic; for scalar uses)
__device__ __forceinline__ float gelu(float x) { return f2u(gelu2(f2(x, x))).x; }

__device__ __forceinline__ float gelu_grad(float x)
{
    const float u = 0.7978845608028654f * fmaf(0.044715f * x, x * x, x);
    const float t = tanh_approx(u);
    return 0.5f * (1.0f + t) + 0.5f * x * (1.0f - t * t) * 0.7978845608028654f * fmaf(0.134145f * x, x, 1.0f);
}

// ---- inputs and output map ------------------------------------------------
// What one sample contributes besides the network: features, ln U, the output
// map's centre (QS) or scale (BW), and whether U <= 1/2.  FP32 from the FP64
// inputs' bits (no FP64 arithmetic): ln chi from the exponent and the leading
// 23 mantissa bits, U truncated to FP32 (relative error < 2^-23).
struct MlpIn {
    float x1, x2, lnu, base;
    bool low;
};

__device__ __forceinline__ MlpIn mlp_input(const MlpView &v, double chi, double u)
{
    MlpIn r;
    const unsigned long long bc = (unsigned long long)__double_as_longlong(chi);
    const int e = (int)((bc >> 52) & 0x7ffu) - 1023;
    const float mc = __uint_as_float(0x3f800000u | (uint32_t)((bc >> 29) & 0x7fffffu));  // [1, 2)
    float lc = fmaf((float)e, 0.6931471805599453f, __logf(mc));
    lc = fminf(fmaxf(lc, v.ln_min), v.ln_max);
    if (e == 1024 || (long long)bc < 0) lc = __int_as_float(0x7fc00000);  // NaN, inf or negative: NaN out
    r.x1 = fmaf(lc - v.ln_min, v.scale, -1.0f);
    const unsigned long long bu = (unsigned long long)__double_as_longlong(u);
    const uint32_t eu = (uint32_t)((bu >> 52) & 0x7ffu);
    float uf = __uint_as_float(((eu - 896u) << 23) | (uint32_t)((bu >> 29) & 0x7fffffu));
    if (eu <= 896u) uf = 1e-38f;  // U below FP32's normal range (U = 0 is not a valid draw)
    r.low = bu <= 0x3FE0000000000000ull;  // U <= 1/2, decided on the FP64 draw
    r.lnu = __logf(uf);
    if (v.proc == QED_PROC_QS) {
        r.x2 = fmaf(2.0f, uf, -1.0f);
        r.base = lc - __logf(1.0f + __expf(lc));
    } else {
        r.x2 = fmaf(4.0f, r.low ? uf : 1.0f - uf, -1.0f);
        r.base = 0.5f * rsqrtf(fmaf(5.333333333333333f, __expf(-lc), 1.0f));
    }
    return r;
}

// network output -> sampled xi (QS: chi_gamma / chi; BW: the electron's chi_- / chi_g)
__device__ __forceinline__ double mlp_output(int proc, float y, const MlpIn &in)
{
    if (proc == QED_PROC_QS) {
        const float l = fmaf(3.0f, in.lnu, y + in.base);
        return (double)(1.0f / (1.0f + __expf(-l)));
    }
    float xs = 1.0f / (1.0f + __expf(4.0f * in.base * y));
    xs = xs > 0.5f ? 0.5f : xs;  // (a NaN y stays NaN)
    return in.low ? (double)xs : 1.0 - (double)xs;  // (1 - xs in FP64 keeps a small xs)
}

// the output y whose map gives xi (the training target of a sample)
__device__ __forceinline__ float mlp_target(int proc, double xi, const MlpIn &in)
{
    if (proc == QED_PROC_QS) return (float)(log(xi) - log1p(-xi)) - fmaf(3.0f, in.lnu, in.base);
    double xs = in.low ? xi : 1.0 - xi;
    xs = xs < 1e-300 ? 1e-300 : (xs > 0.5 ? 0.5 : xs);
    return (float)((log1p(-xs) - log(xs)) / (4.0 * (double)in.base));
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);  // .x = a (low half), .y = b
    return *reinterpret_cast<uint32_t *>(&h);
}

// layer 1 for neurons (k, k + 1), k even: gelu(W1 x + b1) on both lanes.
// w1a / w1b: the coefficients of x1 / x2 as contiguous float arrays.
__device__ __forceinline__ uint64_t layer1_pair(const float *w1a, const float *w1b, const float *b1, int k,
                                                uint64_t x1x1, uint64_t x2x2)
{
    const uint64_t a = *reinterpret_cast<const uint64_t *>(w1a + k);
    const uint64_t b = *reinterpret_cast<const uint64_t *>(w1b + k);
    const uint64_t c = *reinterpret_cast<const uint64_t *>(b1 + k);
    return gelu2(ffma2(a, x1x1, ffma2(b, x2x2, c)));
}

// Stage one network's weights in shared memory: W2 as bf16 rows [n][k] with
// stride kMlpPad, the small layers as float.  All threads of the CTA call it.
struct MlpSmem {
    __nv_bfloat16 w2[kMlpH * kMlpPad];
    alignas(8) float w1a[kMlpH];
    alignas(8) float w1b[kMlpH];
    alignas(8) float b1[kMlpH];
    alignas(8) float b2[kMlpH];
    alignas(8) float w3[kMlpH];
    float b3;
};

__device__ __forceinline__ void mlp_stage(MlpSmem &s, const __nv_bfloat16 *w)
{
    for (int i = threadIdx.x; i < kMlpH * kMlpH; i += blockDim.x)
        s.w2[(i / kMlpH) * kMlpPad + (i % kMlpH)] = w[kOffW2 + i];
    for (int i = threadIdx.x; i < kMlpH; i += blockDim.x) {
        s.w1a[i] = __bfloat162float(w[kOffW1 + 2 * i]);
        s.w1b[i] = __bfloat162float(w[kOffW1 + 2 * i + 1]);
    }
    for (int i = threadIdx.x; i < kMlpH; i += blockDim.x) {
        s.b1[i] = __bfloat162float(w[kOffB1 + i]);
        s.b2[i] = __bfloat162float(w[kOffB2 + i]);
        s.w3[i] = __bfloat162float(w[kOffW3 + i]);
    }
    if (threadIdx.x == 0) s.b3 = __bfloat162float(w[kOffB3]);
}

// Forward pass of 32 samples by one warp (lane l holds sample l's features).
// h1 tile: this warp's bf16 scratch [32][kMlpPad] in shared memory; ybuf: 32
// floats of shared scratch.  All 32 lanes must call it.  Returns y of the lane.
__device__ __forceinline__ float mlp_forward_warp(const MlpSmem &s, __nv_bfloat16 *h1, float *ybuf, float x1,
                                                  float x2)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    // layer 1 on the CUDA cores, rounded to bf16 into the A tile (row = sample)
    uint32_t *row = reinterpret_cast<uint32_t *>(h1 + lane * kMlpPad);
    const uint64_t x1x1 = f2(x1, x1), x2x2 = f2(x2, x2);
#pragma unroll 8
    for (int k = 0; k < kMlpH; k += 2) {
        const float2 g = f2u(layer1_pair(s.w1a, s.w1b, s.b1, k, x1x1, x2x2));
        row[k >> 1] = pack_bf16(g.x, g.y);
    }
    __syncwarp();
    // layer 2 on the tensor cores: Z[32 x 64] = H1[32 x 64] W2^T, in two halves of
    // 32 output neurons; bias, gelu and the layer-3 dot product in the epilogue
    float part[2][2] = {{0.f, 0.f}, {0.f, 0.f}};  // [m-tile][row g / g + 8]
    const uint32_t *A = reinterpret_cast<const uint32_t *>(h1);
    const uint32_t *B = reinterpret_cast<const uint32_t *>(s.w2);
    constexpr int W = kMlpPad / 2;  // 32-bit words per row
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        float acc[2][4][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt)
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.f;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
            uint32_t a[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                const int r0 = (mt * 16 + g) * W + ks * 8 + t;
                a[mt][0] = A[r0];
                a[mt][1] = A[r0 + 8 * W];
                a[mt][2] = A[r0 + 4];
                a[mt][3] = A[r0 + 8 * W + 4];
            }
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int n = half * 32 + nt * 8 + g;
                const uint32_t b0 = B[n * W + ks * 8 + t], b1 = B[n * W + ks * 8 + t + 4];
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    asm volatile(
                        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
                        : "+f"(acc[mt][nt][0]), "+f"(acc[mt][nt][1]), "+f"(acc[mt][nt][2]), "+f"(acc[mt][nt][3])
                        : "r"(a[mt][0]), "r"(a[mt][1]), "r"(a[mt][2]), "r"(a[mt][3]), "r"(b0), "r"(b1));
                }
            }
        }
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                const int n0 = half * 32 + nt * 8 + 2 * t;
                const uint64_t b2 = *reinterpret_cast<const uint64_t *>(s.b2 + n0);
                const uint64_t w3 = *reinterpret_cast<const uint64_t *>(s.w3 + n0);
                const float2 ga = f2u(fmul2(w3, gelu2(fadd2(f2(acc[mt][nt][0], acc[mt][nt][1]), b2))));
                const float2 gb = f2u(fmul2(w3, gelu2(fadd2(f2(acc[mt][nt][2], acc[mt][nt][3]), b2))));
                part[mt][0] += ga.x + ga.y;
                part[mt][1] += gb.x + gb.y;
            }
    }
    // reduce the layer-3 partial sums over the four lanes of a group
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float v = part[mt][h];
            v += __shfl_xor_sync(0xffffffffu, v, 1);
            v += __shfl_xor_sync(0xffffffffu, v, 2);
            part[mt][h] = v;
        }
    if (t == 0) {
        ybuf[g] = part[0][0];
        ybuf[g + 8] = part[0][1];
        ybuf[16 + g] = part[1][0];
        ybuf[16 + g + 8] = part[1][1];
    }
    __syncwarp();
    const float y = ybuf[lane] + s.b3;
    __syncwarp();
    return y;
}

// shared memory of a 256-thread CTA that runs warp-level forward passes
constexpr int kInferThreads = 256;
constexpr int kInferWarps = kInferThreads / 32;

struct InferSmem {
    MlpSmem net;
    __nv_bfloat16 h1[kInferWarps][32 * kMlpPad];
    float y[kInferWarps][32];
};

}  // namespace qed

// the opaque handle of the two networks (QS, BW)
struct qed_mlp {
    int device;
    int64_t max_batch;
    float *master[2];         // FP32 master parameters
    float *adam_m[2], *adam_v[2];
    float *grad[2];           // gradient accumulator (FP32)
    float *part[2];           // per-CTA gradients and loss of the training kernel, [slot][kMlpParams + 1]
    int part_slots;           // CTAs the training kernel may use (one slot each)
    float *loss[2];           // accumulated loss of the last batch
    __nv_bfloat16 *w[2];      // bf16 parameters used by every forward pass
    int64_t step[2];          // Adam step count
    double chi_min[2], chi_max[2];
};

namespace qed {
MlpView mlp_view(const qed_mlp *m, int proc);
}
