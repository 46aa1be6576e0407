// Image loss of the fine-tuning step and its gradient: (1 - lambda) L1 +
// lambda (1 - SSIM), SSIM with an 11x11 Gaussian window (sigma 1.5), zero
// padding, per colour plane (Sec. 4.4 computes the loss "as in" 3DGS).
//
// Two tiled passes over each plane, both with the separable window staged in
// shared memory (a 32 x 16 output tile plus a 5-pixel halo):
//   1. the five windowed moments of x and y -> per-pixel SSIM and the three
//      maps its gradient needs (written to the workspace), plus per-block
//      partial sums of |x - y| and SSIM;
//   2. windowed sums of those maps -> dL/dx per pixel.
// A final one-block kernel adds the partial sums in double in a fixed order,
// so the loss value is deterministic.
#include <cmath>

#include "vbm_internal.h"

namespace vbm {
namespace {

constexpr int kWin = 11;
constexpr int kHalf = 5;
constexpr int kTW = 32, kTH = 16;                  // output tile
constexpr int kSW = kTW + 2 * kHalf, kSH = kTH + 2 * kHalf;
constexpr int kLossThreads = 256;
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;

__constant__ float c_win[kWin];

struct LossWs {
    float *g1, *g2, *g3;
    double *partial;   // [blocks][2]: sum |x - y|, sum ssim
};

__global__ void __launch_bounds__(kLossThreads) k_ssim_fwd(const float *__restrict__ x, const float *__restrict__ y,
                                                          int H, int W, float *__restrict__ g1,
                                                          float *__restrict__ g2, float *__restrict__ g3,
                                                          double *__restrict__ partial)
{
    __shared__ float sx[kSH][kSW], sy[kSH][kSW];
    __shared__ float hs[5][kSH][kTW];
    __shared__ double red[2][kLossThreads];
    const int plane = blockIdx.z;
    const int ox = blockIdx.x * kTW, oy = blockIdx.y * kTH;
    const int64_t base = (int64_t)plane * H * W;
    for (int i = threadIdx.x; i < kSH * kSW; i += blockDim.x) {
        const int r = i / kSW, c = i - r * kSW;
        const int gy = oy + r - kHalf, gx = ox + c - kHalf;
        const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
        sx[r][c] = in ? x[base + (int64_t)gy * W + gx] : 0.f;
        sy[r][c] = in ? y[base + (int64_t)gy * W + gx] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kSH * kTW; i += blockDim.x) {
        const int r = i / kTW, c = i - r * kTW;
        float a = 0.f, b = 0.f, aa = 0.f, bb = 0.f, ab = 0.f;
#pragma unroll
        for (int k = 0; k < kWin; k++) {
            const float w = c_win[k], xv = sx[r][c + k], yv = sy[r][c + k];
            a += w * xv;
            b += w * yv;
            aa += w * xv * xv;
            bb += w * yv * yv;
            ab += w * xv * yv;
        }
        hs[0][r][c] = a; hs[1][r][c] = b; hs[2][r][c] = aa; hs[3][r][c] = bb; hs[4][r][c] = ab;
    }
    __syncthreads();
    double l1 = 0.0, ss = 0.0;
    for (int i = threadIdx.x; i < kTH * kTW; i += blockDim.x) {
        const int r = i / kTW, c = i - r * kTW;
        const int gy = oy + r, gx = ox + c;
        if (gy >= H || gx >= W) continue;
        float mx = 0.f, my = 0.f, exx = 0.f, eyy = 0.f, exy = 0.f;
#pragma unroll
        for (int k = 0; k < kWin; k++) {
            const float w = c_win[k];
            mx += w * hs[0][r + k][c];
            my += w * hs[1][r + k][c];
            exx += w * hs[2][r + k][c];
            eyy += w * hs[3][r + k][c];
            exy += w * hs[4][r + k][c];
        }
        const float vx = exx - mx * mx, vy = eyy - my * my, cxy = exy - mx * my;
        const float A1 = 2.f * mx * my + kC1, A2 = 2.f * cxy + kC2;
        const float B1 = mx * mx + my * my + kC1, B2 = vx + vy + kC2;
        const float iB1 = 1.f / B1, iB2 = 1.f / B2;
        const float ssim = A1 * A2 * iB1 * iB2;
        const int64_t e = base + (int64_t)gy * W + gx;
        g1[e] = 2.f * my * (A2 - A1) * iB1 * iB2 - 2.f * mx * ssim * (iB1 - iB2);
        g2[e] = -ssim * iB2;
        g3[e] = 2.f * A1 * iB1 * iB2;
        l1 += fabs((double)sx[r + kHalf][c + kHalf] - (double)sy[r + kHalf][c + kHalf]);
        ss += ssim;
    }
    red[0][threadIdx.x] = l1;
    red[1][threadIdx.x] = ss;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < (unsigned)off) {
            red[0][threadIdx.x] += red[0][threadIdx.x + off];
            red[1][threadIdx.x] += red[1][threadIdx.x + off];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int64_t b = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        partial[2 * b] = red[0][0];
        partial[2 * b + 1] = red[1][0];
    }
}

__global__ void __launch_bounds__(kLossThreads) k_ssim_bwd(const float *__restrict__ x, const float *__restrict__ y,
                                                          int H, int W, const float *__restrict__ g1,
                                                          const float *__restrict__ g2, const float *__restrict__ g3,
                                                          float lambda, float scale, float *__restrict__ dx)
{
    __shared__ float s[3][kSH][kSW];
    __shared__ float hs[3][kSH][kTW];
    const int plane = blockIdx.z;
    const int ox = blockIdx.x * kTW, oy = blockIdx.y * kTH;
    const int64_t base = (int64_t)plane * H * W;
    for (int i = threadIdx.x; i < kSH * kSW; i += blockDim.x) {
        const int r = i / kSW, c = i - r * kSW;
        const int gy = oy + r - kHalf, gx = ox + c - kHalf;
        const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
        const int64_t e = base + (int64_t)gy * W + gx;
        s[0][r][c] = in ? g1[e] : 0.f;
        s[1][r][c] = in ? g2[e] : 0.f;
        s[2][r][c] = in ? g3[e] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kSH * kTW; i += blockDim.x) {
        const int r = i / kTW, c = i - r * kTW;
        float a = 0.f, b = 0.f, d = 0.f;
#pragma unroll
        for (int k = 0; k < kWin; k++) {
            const float w = c_win[k];
            a += w * s[0][r][c + k];
            b += w * s[1][r][c + k];
            d += w * s[2][r][c + k];
        }
        hs[0][r][c] = a; hs[1][r][c] = b; hs[2][r][c] = d;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kTH * kTW; i += blockDim.x) {
        const int r = i / kTW, c = i - r * kTW;
        const int gy = oy + r, gx = ox + c;
        if (gy >= H || gx >= W) continue;
        float a = 0.f, b = 0.f, d = 0.f;
#pragma unroll
        for (int k = 0; k < kWin; k++) {
            const float w = c_win[k];
            a += w * hs[0][r + k][c];
            b += w * hs[1][r + k][c];
            d += w * hs[2][r + k][c];
        }
        const int64_t e = base + (int64_t)gy * W + gx;
        const float xv = x[e], yv = y[e];
        const float diff = xv - yv;
        const float sgn = diff > 0.f ? 1.f : (diff < 0.f ? -1.f : 0.f);
        const float dssim = a + 2.f * xv * b + yv * d;
        dx[e] = scale * ((1.f - lambda) * sgn - lambda * dssim);
    }
}

__global__ void k_loss_final(const double *__restrict__ partial, int64_t blocks, double n_elem, double lambda,
                             double scale, double *__restrict__ loss, int accumulate)
{
    __shared__ double red[2][256];
    double a = 0.0, b = 0.0;
    for (int64_t i = threadIdx.x; i < blocks; i += blockDim.x) {
        a += partial[2 * i];
        b += partial[2 * i + 1];
    }
    red[0][threadIdx.x] = a;
    red[1][threadIdx.x] = b;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < (unsigned)off) {
            red[0][threadIdx.x] += red[0][threadIdx.x + off];
            red[1][threadIdx.x] += red[1][threadIdx.x + off];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double L = scale * ((1.0 - lambda) * red[0][0] + lambda * (n_elem - red[1][0]));
        *loss = accumulate ? *loss + L : L;
    }
}

bool g_win_ready = false;

vbm_status ensure_window()
{
    if (g_win_ready) return VBM_OK;
    double g[kWin], s = 0.0;
    for (int i = 0; i < kWin; i++) {
        const double d = i - kHalf;
        g[i] = std::exp(-d * d / (2.0 * 1.5 * 1.5));
        s += g[i];
    }
    float w[kWin];
    for (int i = 0; i < kWin; i++) w[i] = (float)(g[i] / s);
    VBM_CUDA(cudaMemcpyToSymbol(c_win, w, sizeof(w)));
    g_win_ready = true;
    return VBM_OK;
}

size_t loss_blocks(int n_images, int H, int W)
{
    return (size_t)((W + kTW - 1) / kTW) * ((H + kTH - 1) / kTH) * (size_t)n_images * 3;
}

}  // namespace

size_t loss_workspace_bytes(int n_images, int H, int W)
{
    const size_t n = (size_t)n_images * 3 * H * W;
    size_t bytes = 3 * n * sizeof(float);
    bytes = (bytes + 255) / 256 * 256;
    return bytes + loss_blocks(n_images, H, W) * 2 * sizeof(double);
}

vbm_status loss_fwd_bwd(const float *img, const float *target, int n_images, int H, int W, float lambda,
                        double scale, double *loss, int accumulate, float *dimg, void *ws, cudaStream_t st)
{
    vbm_status s = ensure_window();
    if (s != VBM_OK) return s;
    const size_t n = (size_t)n_images * 3 * H * W;
    char *p = (char *)ws;
    float *g1 = (float *)p, *g2 = g1 + n, *g3 = g2 + n;
    size_t off = (3 * n * sizeof(float) + 255) / 256 * 256;
    double *partial = (double *)(p + off);
    dim3 grid((W + kTW - 1) / kTW, (H + kTH - 1) / kTH, n_images * 3);
    k_ssim_fwd<<<grid, kLossThreads, 0, st>>>(img, target, H, W, g1, g2, g3, partial);
    VBM_LAUNCH("ssim_fwd");
    k_ssim_bwd<<<grid, kLossThreads, 0, st>>>(img, target, H, W, g1, g2, g3, lambda, (float)scale, dimg);
    VBM_LAUNCH("ssim_bwd");
    k_loss_final<<<1, 256, 0, st>>>(partial, (int64_t)grid.x * grid.y * grid.z, (double)n, (double)lambda, scale,
                                    loss, accumulate);
    VBM_LAUNCH("loss_final");
    note_launches(3);
    return VBM_OK;
}

}  // namespace vbm
