// Fused Adam update of the Gaussian parameters (Sec. 5.2 uses Adam).
//
// One thread per scalar of P[14][stride] (first n columns), reading p, g, m,
// v and writing p, m, v: 28 bytes of HBM traffic per scalar, coalesced.  The
// step counter lives on the device so the update can be replayed from a CUDA
// graph: a one-thread kernel increments it, the update reads it.
#include <cmath>

#include "vbm_internal.h"

namespace vbm {
namespace {

__global__ void k_step_inc(int32_t *step)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *step += 1;
}

__global__ void k_adam(float *__restrict__ P, const float *__restrict__ G, float *__restrict__ M,
                       float *__restrict__ V, int64_t n, int64_t stride, const int32_t *__restrict__ step,
                       float lr0, float lr1, float lr2, float lr3, float lr4, float beta1, float beta2, float eps,
                       uint32_t *__restrict__ nonfinite)
{
    // the bias corrections are the same for every scalar: one thread of the
    // block evaluates them
    __shared__ float s_bc[2];
    if (threadIdx.x == 0) {
        const int t = *step;
        s_bc[0] = 1.f - powf(beta1, (float)t);
        s_bc[1] = 1.f - powf(beta2, (float)t);
    }
    __syncthreads();
    const int row = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float lr = row < 3 ? lr0 : row < 6 ? lr1 : row < 10 ? lr2 : row < 11 ? lr3 : lr4;
    const float bc1 = s_bc[0];
    const float bc2 = s_bc[1];
    const int64_t e = row * stride + i;
    const float g = G[e];
    if (!isfinite(g)) {
        if (nonfinite) atomicAdd(nonfinite, 1u);
        return;
    }
    const float m = beta1 * M[e] + (1.f - beta1) * g;
    const float v = beta2 * V[e] + (1.f - beta2) * g * g;
    M[e] = m;
    V[e] = v;
    const float mhat = m / bc1;
    const float vhat = v / bc2;
    P[e] -= lr * mhat / (sqrtf(vhat) + eps);
}

}  // namespace

vbm_status adam_step(float *P, const float *G, float *M, float *V, int64_t n, int64_t stride, int32_t *step,
                     const float lrs[5], float beta1, float beta2, float eps, uint32_t *nonfinite, cudaStream_t st)
{
    k_step_inc<<<1, 32, 0, st>>>(step);
    VBM_LAUNCH("adam_step_inc");
    note_launches(1);
    if (n == 0) return VBM_OK;
    dim3 grid((unsigned)((n + 255) / 256), 14);
    k_adam<<<grid, 256, 0, st>>>(P, G, M, V, n, stride, step, lrs[0], lrs[1], lrs[2], lrs[3], lrs[4], beta1, beta2,
                                 eps, nonfinite);
    VBM_LAUNCH("adam");
    note_launches(1);
    return VBM_OK;
}

}  // namespace vbm
