// measure.cu -- standalone throughput probes: the FP64 peak against which the
// FP64 evolution kernel (bound by GB300's FP64 pipe) is judged, measured by a
// kernel that does nothing but dependent chains of fused multiply-adds; the
// special-function unit's tanh.approx.f32 rate, which bounds the learned
// sampler's GELUs; and an evaluation of the rate lookups' FP64 logarithm and
// exponential beside the CUDA library's, for their accuracy checks.
#include "fp64_math.cuh"
#include "launch.cuh"
#include "mlp.cuh"

namespace qed {

constexpr int kProbeChains = 8;  // independent chains per thread (hide the FMA latency)

__global__ void __launch_bounds__(256) fp64_fma_kernel(int64_t iters, double a, double b, double *sink)
{
    double x[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = (double)(threadIdx.x + c) * 1e-3;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += x[c];
    if (s == 1234.5678) sink[0] = s;  // keeps the chains alive; never true for these inputs
}

// dependent chains x <- a tanh(x) + b: one tanh.approx.f32 and one FMA per step
__global__ void __launch_bounds__(256) tanh_kernel(int64_t iters, float a, float b, double *sink)
{
    float x[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) x[c] = fmaf(a, tanh_approx(x[c]), b);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += x[c];
    if (s == 1234.5678f) sink[0] = s;  // keeps the chains alive; never true for these inputs
}

// one warm-up launch, then one timed launch of `kernel` on `grid` CTAs of 256;
// *ops_per_s = grid x 256 x kProbeChains x iters / time
template <typename A>
static qed_status time_probe(void (*kernel)(int64_t, A, A, double *), int64_t iters, A a, A b, int grid,
                             double *d_sink, double *ops_per_s, float *ms_out, cudaStream_t st)
{
    cudaEvent_t e0, e1;
    QED_CUDA_TRY(cudaEventCreate(&e0));
    QED_CUDA_TRY(cudaEventCreate(&e1));
    kernel<<<grid, 256, 0, st>>>(iters / 10 + 1, a, b, d_sink);  // warm-up
    cudaEventRecord(e0, st);
    kernel<<<grid, 256, 0, st>>>(iters, a, b, d_sink);
    cudaEventRecord(e1, st);
    const cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) QED_FAIL(QED_ERR_CUDA, "probe failed: %s", cudaGetErrorString(e));
    *ops_per_s = (double)grid * 256.0 * kProbeChains * (double)iters / (ms * 1e-3);
    if (ms_out) *ms_out = ms;
    return QED_OK;
}

}  // namespace qed

using namespace qed;

extern "C" qed_status qed_probe_tanh(int64_t iters, int32_t ctas_per_sm, double *d_sink, double *tanh_per_s,
                                     float *ms_out, void *stream)
{
    clear_error();
    if (iters <= 0 || ctas_per_sm <= 0 || ctas_per_sm > 32 || !d_sink || !tanh_per_s)
        QED_FAIL(QED_ERR_INVALID_ARG, "bad probe arguments");
    return time_probe(tanh_kernel, iters, 0.5f, 0.5f, sm_count() * ctas_per_sm, d_sink, tanh_per_s, ms_out,
                      as_stream(stream));
}

extern "C" qed_status qed_probe_fp64_fma(int64_t iters, int32_t ctas_per_sm, double *d_sink, double *fma_per_s,
                                         float *ms_out, void *stream)
{
    clear_error();
    if (iters <= 0 || ctas_per_sm <= 0 || ctas_per_sm > 32 || !d_sink || !fma_per_s)
        QED_FAIL(QED_ERR_INVALID_ARG, "bad probe arguments");
    return time_probe(fp64_fma_kernel, iters, 0.999999, 1e-7, sm_count() * ctas_per_sm, d_sink, fma_per_s, ms_out,
                      as_stream(stream));
}

namespace qed {

__global__ void fp64_logexp_kernel(const double *x, int64_t n, double *out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = x[i];
        out[i] = log_tang(v);
        out[n + i] = exp_tang(v);
        out[2 * n + i] = log(v);
        out[3 * n + i] = exp(v);
    }
}

}  // namespace qed

extern "C" qed_status qed_probe_fp64_logexp(const double *d_x, int64_t n, double *d_out, void *stream)
{
    clear_error();
    if (n < 0) QED_FAIL(QED_ERR_INVALID_ARG, "n < 0");
    if (n == 0) return QED_OK;
    if (!d_x || !d_out) QED_FAIL(QED_ERR_INVALID_ARG, "a pointer is NULL");
    if (n > ((int64_t)1 << 40)) QED_FAIL(QED_ERR_INVALID_ARG, "n > 2^40");
    const int64_t want = (n + 255) / 256, cap = 8 * (int64_t)sm_count();
    fp64_logexp_kernel<<<(int)(want < cap ? want : cap), 256, 0, as_stream(stream)>>>(d_x, n, d_out);
    QED_LAUNCH_CHECK();
    return QED_OK;
}
