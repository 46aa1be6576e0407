// Fused Adam update of the Gaussian parameters (Sec. 5.2 uses Adam).
//
// Updates the first n columns of P[14][stride], reading p, g, m, v and
// writing p, m, v: 28 bytes of HBM traffic per scalar, coalesced; four
// scalars per thread when the rows are packed (stride == n), one otherwise.  The
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

// the bias corrections are the same for every scalar: one thread of the block
// evaluates them
__device__ __forceinline__ void bias_corrections(float *s_bc, const int32_t *step, float beta1, float beta2)
{
    if (threadIdx.x == 0) {
        const int t = *step;
        const float2 bc = adam_bias_corrections(t, beta1, beta2);
        s_bc[0] = bc.x;
        s_bc[1] = bc.y;
    }
    __syncthreads();
}

// Rows packed back to back (stride == n): the 14 n scalars are one array,
// four per thread with 16-byte loads and stores; each scalar takes its own
// row's learning rate (a quad may cross rows).
__global__ void k_adam_flat(float *__restrict__ P, const float *__restrict__ G, float *__restrict__ M,
                            float *__restrict__ V, int64_t n, const int32_t *__restrict__ step, float lr0, float lr1,
                            float lr2, float lr3, float lr4, float beta1, float beta2, float eps,
                            uint32_t *__restrict__ nonfinite)
{
    __shared__ float s_bc[2];
    bias_corrections(s_bc, step, beta1, beta2);
    const int64_t total = 14 * n;
    const int64_t e0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (e0 >= total) return;
    const float bc1 = s_bc[0];
    const float bc2 = s_bc[1];
    int row = (int)(e0 / n);
    int64_t row_end = (int64_t)(row + 1) * n;
    uint32_t bad = 0;
    if (e0 + 4 <= total) {
        float4 g4 = *reinterpret_cast<const float4 *>(G + e0);
        float4 p4 = *reinterpret_cast<const float4 *>(P + e0);
        float4 m4 = *reinterpret_cast<const float4 *>(M + e0);
        float4 v4 = *reinterpret_cast<const float4 *>(V + e0);
        float *g = &g4.x, *p = &p4.x, *m = &m4.x, *v = &v4.x;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            while (e0 + k >= row_end) {
                ++row;
                row_end += n;
            }
            bad += !adam_elem(p[k], m[k], v[k], g[k], adam_row_lr(row, lr0, lr1, lr2, lr3, lr4), beta1, beta2, eps, bc1,
                              bc2);
        }
        *reinterpret_cast<float4 *>(P + e0) = p4;
        *reinterpret_cast<float4 *>(M + e0) = m4;
        *reinterpret_cast<float4 *>(V + e0) = v4;
    } else {
        for (int64_t e = e0; e < total; ++e) {
            while (e >= row_end) {
                ++row;
                row_end += n;
            }
            float p = P[e], m = M[e], v = V[e];
            if (!adam_elem(p, m, v, G[e], adam_row_lr(row, lr0, lr1, lr2, lr3, lr4), beta1, beta2, eps, bc1, bc2)) {
                ++bad;
                continue;
            }
            P[e] = p;
            M[e] = m;
            V[e] = v;
        }
    }
    if (bad && nonfinite) atomicAdd(nonfinite, bad);
}

// Rows with padding (stride > n) or unaligned pointers: one scalar per
// thread, one grid row per parameter row.
__global__ void k_adam_rows(float *__restrict__ P, const float *__restrict__ G, float *__restrict__ M,
                            float *__restrict__ V, int64_t n, int64_t stride, const int32_t *__restrict__ step,
                            float lr0, float lr1, float lr2, float lr3, float lr4, float beta1, float beta2, float eps,
                            uint32_t *__restrict__ nonfinite)
{
    __shared__ float s_bc[2];
    bias_corrections(s_bc, step, beta1, beta2);
    const int row = blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t e = row * stride + i;
    float p = P[e], m = M[e], v = V[e];
    if (!adam_elem(p, m, v, G[e], adam_row_lr(row, lr0, lr1, lr2, lr3, lr4), beta1, beta2, eps, s_bc[0], s_bc[1])) {
        if (nonfinite) atomicAdd(nonfinite, 1u);
        return;
    }
    P[e] = p;
    M[e] = m;
    V[e] = v;
}

}  // namespace

vbm_status adam_step_inc(int32_t *step, cudaStream_t st)
{
    k_step_inc<<<1, 32, 0, st>>>(step);
    VBM_LAUNCH("adam_step_inc");
    note_launches(1);
    return VBM_OK;
}

vbm_status adam_step(float *P, const float *G, float *M, float *V, int64_t n, int64_t stride, int32_t *step,
                     const float lrs[5], float beta1, float beta2, float eps, uint32_t *nonfinite, cudaStream_t st)
{
    vbm_status s = adam_step_inc(step, st);
    if (s != VBM_OK) return s;
    if (n == 0) return VBM_OK;
    const bool flat = stride == n && ((reinterpret_cast<uintptr_t>(P) | reinterpret_cast<uintptr_t>(G) |
                                       reinterpret_cast<uintptr_t>(M) | reinterpret_cast<uintptr_t>(V)) & 15) == 0;
    if (flat) {
        const int64_t quads = (14 * n + 3) / 4;
        k_adam_flat<<<(unsigned)((quads + 255) / 256), 256, 0, st>>>(P, G, M, V, n, step, lrs[0], lrs[1], lrs[2],
                                                                     lrs[3], lrs[4], beta1, beta2, eps, nonfinite);
    } else {
        dim3 grid((unsigned)((n + 255) / 256), 14);
        k_adam_rows<<<grid, 256, 0, st>>>(P, G, M, V, n, stride, step, lrs[0], lrs[1], lrs[2], lrs[3], lrs[4], beta1,
                                          beta2, eps, nonfinite);
    }
    VBM_LAUNCH("adam");
    note_launches(1);
    return VBM_OK;
}

}  // namespace vbm
