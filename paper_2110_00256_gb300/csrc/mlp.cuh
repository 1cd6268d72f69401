// mlp.cuh -- the learned inverse-CDF sampler: a 2-64-64-1 GELU network per
// process (QS: ln xi - 3 ln U; BW: the folded pair-split fraction), bfloat16
// weights, FP32 accumulation, the 64x64 layer on the tensor cores
// (mma.sync m16n8k16 bf16 -> f32).  The paper has no learned sampler: this
// stands in for the 2-D inverse-CDF tables of §3.1 and §3.2.
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
    float ln_min, scale, chi_min, chi_max;
    int proc;                // QED_PROC_QS or QED_PROC_BW
};

__device__ __forceinline__ float tanh_approx(float x)
{
    float y;
    asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// gelu(x) = x/2 (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3)))  (Hendrycks & Gimpel),
// evaluated as h + h tanh(u) with h = x/2, u = x (sqrt(2/pi) + sqrt(2/pi) 0.044715 x^2):
// six instructions, the GELUs being what bounds the network's throughput
__device__ __forceinline__ float gelu(float x)
{
    const float u = x * fmaf(0.035677408136300125f, x * x, 0.7978845608028654f);
    const float h = 0.5f * x;
    return fmaf(h, tanh_approx(u), h);
}

__device__ __forceinline__ float gelu_grad(float x)
{
    const float u = 0.7978845608028654f * fmaf(0.044715f * x, x * x, x);
    const float t = tanh_approx(u);
    return 0.5f * (1.0f + t) + 0.5f * x * (1.0f - t * t) * 0.7978845608028654f * fmaf(0.134145f * x, x, 1.0f);
}

// features of one sample (see the parameter layout above)
// (FP32 arithmetic: the network itself works to bf16 precision)
__device__ __forceinline__ void mlp_features(const MlpView &v, double chi, double u, float &x1, float &x2)
{
    float c = (float)chi;
    c = c < v.chi_min ? v.chi_min : (c > v.chi_max ? v.chi_max : c);
    x1 = (logf(c) - v.ln_min) * v.scale - 1.0f;
    const double up = v.proc == QED_PROC_QS ? u : 2.0 * (u < 1.0 - u ? u : 1.0 - u);
    x2 = (float)(2.0 * up - 1.0);
}

// network output -> sampled xi.  QS: xi = exp(min(y + 3 ln U, 0)).  BW: the
// electron's fraction chi_- / chi_g, from the folded fraction clamp(y, 0, 1/2)
// of the lepton that U selects (U <= 1/2: electron), as in the table path.
__device__ __forceinline__ double mlp_output(int proc, float y, double u)
{
    if (proc == QED_PROC_QS) {
        const float l = fmaf(3.0f, logf((float)u), y);
        return (double)expf(l > 0.0f ? 0.0f : l);
    }
    double xs = y < 0.0f ? 0.0 : (y > 0.5f ? 0.5 : (double)y);
    return u <= 0.5 ? xs : 1.0 - xs;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);  // .x = a (low half), .y = b
    return *reinterpret_cast<uint32_t *>(&h);
}

// Stage one network's weights in shared memory: W2 as bf16 rows [n][k] with
// stride kMlpPad, the small layers as float.  All threads of the CTA call it.
struct MlpSmem {
    __nv_bfloat16 w2[kMlpH * kMlpPad];
    float w1[kMlpH * 2], b1[kMlpH], b2[kMlpH], w3[kMlpH];
    float b3;
};

__device__ __forceinline__ void mlp_stage(MlpSmem &s, const __nv_bfloat16 *w)
{
    for (int i = threadIdx.x; i < kMlpH * kMlpH; i += blockDim.x)
        s.w2[(i / kMlpH) * kMlpPad + (i % kMlpH)] = w[kOffW2 + i];
    for (int i = threadIdx.x; i < kMlpH * 2; i += blockDim.x) s.w1[i] = __bfloat162float(w[kOffW1 + i]);
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
#pragma unroll 8
    for (int k = 0; k < kMlpH; k += 2) {
        const float a = gelu(fmaf(s.w1[2 * k], x1, fmaf(s.w1[2 * k + 1], x2, s.b1[k])));
        const float b = gelu(fmaf(s.w1[2 * k + 2], x1, fmaf(s.w1[2 * k + 3], x2, s.b1[k + 1])));
        row[k >> 1] = pack_bf16(a, b);
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
                part[mt][0] += s.w3[n0] * gelu(acc[mt][nt][0] + s.b2[n0]) +
                               s.w3[n0 + 1] * gelu(acc[mt][nt][1] + s.b2[n0 + 1]);
                part[mt][1] += s.w3[n0] * gelu(acc[mt][nt][2] + s.b2[n0]) +
                               s.w3[n0 + 1] * gelu(acc[mt][nt][3] + s.b2[n0 + 1]);
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
    float *loss[2];           // accumulated loss of the last batch
    __nv_bfloat16 *w[2];      // bf16 parameters used by every forward pass
    int64_t step[2];          // Adam step count
    double chi_min[2], chi_max[2];
};

namespace qed {
MlpView mlp_view(const qed_mlp *m, int proc);
}
