// Throughput probes for the roofline denominators of the compositing kernels:
// dependent chains of scalar FP32 FMAs, of packed FP32x2 FMAs, and of ex2
// (the special-function unit's base-2 exponential), each thread running
// kChains independent chains so that the pipes, not the latencies, bound the
// rate.  Timed by the caller with CUDA events around one launch.
#include "vbm_internal.h"

namespace vbm {
namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

__global__ void __launch_bounds__(256) k_peak_ffma(int iters, float b, float c, float *out)
{
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) a[k] = (float)(threadIdx.x + k) * 1e-3f;
    for (int i = 0; i < iters; i += kUnroll) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++)
#pragma unroll
            for (int k = 0; k < kChains; k++) a[k] = fmaf(a[k], b, c);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += a[k];
    if (s == 12345.f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains live
}

__global__ void __launch_bounds__(256) k_peak_ffma2(int iters, float b, float c, float *out)
{
    float2 a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) a[k] = make_float2((float)(threadIdx.x + k) * 1e-3f, (float)k * 1e-3f);
    const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
    for (int i = 0; i < iters; i += kUnroll) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++)
#pragma unroll
            for (int k = 0; k < kChains; k++) a[k] = __ffma2_rn(a[k], b2, c2);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += a[k].x + a[k].y;
    if (s == 12345.f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// x <- 0.25 - 0.5 * 2^x keeps x in [-0.25, -0.17]: one ex2 and one FMA per link
__global__ void __launch_bounds__(256) k_peak_ex2(int iters, float *out)
{
    float a[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) a[k] = -0.2f - (float)k * 1e-3f;
    for (int i = 0; i < iters; i += kUnroll) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++)
#pragma unroll
            for (int k = 0; k < kChains; k++) a[k] = fmaf(ex2_approx(a[k]), -0.5f, 0.25f);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += a[k];
    if (s == 12345.f) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace vbm

using namespace vbm;

extern "C" {

vbm_status vbm_peak_probe(int32_t kind, int32_t blocks, int32_t iters, float *d_out, double *ops, void *stream)
{
    VBM_ARG(kind >= 0 && kind <= 2, "kind must be 0 (FP32 FMA), 1 (FP32x2 FMA) or 2 (ex2)");
    VBM_ARG(blocks > 0 && iters > 0 && iters % kUnroll == 0, "blocks > 0, iters a positive multiple of 16");
    VBM_ARG(d_out && ops, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    const double lanes = (double)blocks * 256 * (double)iters * kChains;
    if (kind == 0) {
        k_peak_ffma<<<blocks, 256, 0, st>>>(iters, 0.99991f, 1e-4f, d_out);
        *ops = 2.0 * lanes;                     // FLOP
    } else if (kind == 1) {
        k_peak_ffma2<<<blocks, 256, 0, st>>>(iters, 0.99991f, 1e-4f, d_out);
        *ops = 4.0 * lanes;                     // FLOP: two FMAs per packed instruction
    } else {
        k_peak_ex2<<<blocks, 256, 0, st>>>(iters, d_out);
        *ops = lanes;                           // ex2 evaluations
    }
    VBM_LAUNCH("peak_probe");
    note_launches(1);
    return VBM_OK;
}

}  // extern "C"
