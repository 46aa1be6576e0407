// Image loss of the fine-tuning step and its gradient: (1 - lambda) L1 +
// lambda (1 - SSIM), SSIM with an 11x11 Gaussian window (sigma 1.5), zero
// padding, per colour plane (Sec. 4.4 computes the loss "as in" 3DGS).
//
// Two tiled passes over each plane, each staging a 32 x 32 output tile plus a
// 5-pixel halo in shared memory and applying the separable window as a
// horizontal then a vertical pass:
//   1. the five windowed moments of x and y -> per-pixel SSIM and the three
//      maps its gradient needs (written to the workspace as a float2 and a
//      float plane), plus per-block sums of |x - y| and SSIM;
//   2. windowed sums of those maps -> dL/dx per pixel.
// In both passes a thread slides the window along a row segment (horizontal)
// or a column segment (vertical) held in registers, so each staged value is
// read from shared memory once per pass; the moment pairs (x, y), (x^2, y^2)
// and the map pair (g1, g2) are accumulated with packed FP32x2 FMAs.
// The first block of pass 2 adds pass 1's per-block sums in double in a fixed
// order (they are complete when pass 2 starts), so the loss value is
// deterministic and needs no launch of its own.
#include <cmath>

#include <mutex>

#include "vbm_internal.h"

namespace vbm {
namespace {

constexpr int kWin = 11;
constexpr int kHalf = 5;
constexpr int kTW = 32, kTH = 32;                  // output tile
constexpr int kSW = kTW + 2 * kHalf, kSH = kTH + 2 * kHalf;
constexpr int kSWP = kSW + 2;                      // padded row of the staged tile (zero-filled)
constexpr int kHP = kTW + 1;                       // padded row of the horizontal sums
constexpr int kSeg = 11, kSegs = 3;                // horizontal: 3 segments of <= 11 outputs per row
constexpr int kVRows = 8;                          // vertical: 8 outputs per column segment
constexpr int kLossThreads = 128;
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;
static_assert(kSegs * kSeg >= kTW && kSH * kSegs <= kLossThreads, "horizontal tasks");
static_assert(kTW * (kTH / kVRows) == kLossThreads, "vertical tasks");
static_assert((kSegs - 1) * kSeg + kSeg + kWin - 1 <= kSWP, "staged row covers the last segment");

__constant__ float c_win[kWin];

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// Hardware reciprocal (one MUFU operation, relative error of the order of one
// FP32 rounding); its operands here are >= C1 = 1e-4, far from subnormals.
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Stage plane values (or value pairs) of rows [oy - 5, oy + kTH + 5) and columns
// [ox - 5, ox + kTW + 5) into s[kSH][kSWP]; outside the image (and the pad
// columns) they are zero.  Warp w stages rows w, w + 4, ...: lane l loads
// columns l and 32 + l of each, so every load instruction reads consecutive
// pixels of one row and the index arithmetic is per row, not per value.
// Every load of a thread is issued before the first store.
constexpr int kLossWarps = kLossThreads / 32;
constexpr int kStageRows = (kSH + kLossWarps - 1) / kLossWarps;
static_assert(kSWP > 32 && kSWP <= 64, "a staged row is two loads per lane");

template <typename T, typename F>
__device__ __forceinline__ void stage_tile(T (*s)[kSWP], int ox, int oy, int H, int W, F load)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gx0 = ox - kHalf + lane, gx1 = gx0 + 32;
    const bool in0 = gx0 >= 0 && gx0 < W;
    const bool in1 = lane < kSW - 32 && gx1 >= 0 && gx1 < W;
    T v0[kStageRows], v1[kStageRows];
#pragma unroll
    for (int k = 0; k < kStageRows; k++) {
        const int r = warp + k * kLossWarps;
        const int gy = oy + r - kHalf;
        const bool rin = r < kSH && gy >= 0 && gy < H;
        const int64_t row = (int64_t)gy * W;
        v0[k] = load(rin && in0, row + gx0);
        v1[k] = load(rin && in1, row + gx1);
    }
#pragma unroll
    for (int k = 0; k < kStageRows; k++) {
        const int r = warp + k * kLossWarps;
        if (r < kSH) {
            s[r][lane] = v0[k];
            if (lane < kSWP - 32) s[r][32 + lane] = v1[k];
        }
    }
}

__global__ void __launch_bounds__(kLossThreads) k_ssim_fwd(const float *__restrict__ x, const float *__restrict__ y,
                                                          int H, int W, float2 *__restrict__ g12,
                                                          float *__restrict__ g3, double *__restrict__ partial)
{
    __shared__ __align__(16) float2 sxy[kSH][kSWP];
    // horizontal sums of (x, y), (x^2, y^2) and x y; rows padded by one
    // element so the horizontal pass's lanes (11 rows at the same column)
    // write to different banks
    __shared__ __align__(16) float2 hm[kSH][kHP];
    __shared__ __align__(16) float2 hq[kSH][kHP];
    __shared__ float hp[kSH][kHP];
    __shared__ float red[2][kLossThreads / 32];
    const int plane = blockIdx.z;
    const int ox = blockIdx.x * kTW, oy = blockIdx.y * kTH;
    const int64_t base = (int64_t)plane * H * W;
    const float *xp = x + base, *yp = y + base;
    stage_tile(sxy, ox, oy, H, W, [&](bool in, int64_t e) {
        return in ? make_float2(xp[e], yp[e]) : make_float2(0.f, 0.f);
    });
    __syncthreads();
    const int t = threadIdx.x;
    if (t < kSH * kSegs) {
        const int r = t / kSegs, c0 = (t - r * kSegs) * kSeg;
        float2 v[kSeg + kWin - 1], sq[kSeg + kWin - 1];
        float pr[kSeg + kWin - 1];
#pragma unroll
        for (int j = 0; j < kSeg + kWin - 1; j++) {
            v[j] = sxy[r][c0 + j];
            sq[j] = __fmul2_rn(v[j], v[j]);
            pr[j] = v[j].x * v[j].y;
        }
#pragma unroll
        for (int o = 0; o < kSeg; o++) {
            float2 m = make_float2(0.f, 0.f), q = m;
            float p = 0.f;
#pragma unroll
            for (int k = 0; k < kWin; k++) {
                const float w = c_win[k];
                m = __ffma2_rn(f2(w), v[o + k], m);
                q = __ffma2_rn(f2(w), sq[o + k], q);
                p = fmaf(w, pr[o + k], p);
            }
            if (c0 + o < kTW) {
                hm[r][c0 + o] = m;
                hq[r][c0 + o] = q;
                hp[r][c0 + o] = p;
            }
        }
    }
    __syncthreads();
    const int c = t & 31, r0 = (t >> 5) * kVRows;
    float l1 = 0.f, ss = 0.f;
    float2 m_in[kVRows + kWin - 1], q_in[kVRows + kWin - 1];
    float p_in[kVRows + kWin - 1];
#pragma unroll
    for (int j = 0; j < kVRows + kWin - 1; j++) {
        m_in[j] = hm[r0 + j][c];
        q_in[j] = hq[r0 + j][c];
        p_in[j] = hp[r0 + j][c];
    }
    const int gx = ox + c;
#pragma unroll
    for (int o = 0; o < kVRows; o++) {
        float2 m = make_float2(0.f, 0.f), q = m;
        float p = 0.f;
#pragma unroll
        for (int k = 0; k < kWin; k++) {
            const float w = c_win[k];
            m = __ffma2_rn(f2(w), m_in[o + k], m);
            q = __ffma2_rn(f2(w), q_in[o + k], q);
            p = fmaf(w, p_in[o + k], p);
        }
        const int gy = oy + r0 + o;
        if (gy >= H || gx >= W) continue;
        const float mx = m.x, my = m.y;
        const float vx = q.x - mx * mx, vy = q.y - my * my, cxy = p - mx * my;
        const float A1 = 2.f * mx * my + kC1, A2 = 2.f * cxy + kC2;
        const float B1 = mx * mx + my * my + kC1, B2 = vx + vy + kC2;
        const float iB1 = rcp_approx(B1), iB2 = rcp_approx(B2);
        const float ssim = A1 * A2 * iB1 * iB2;
        const int64_t e = base + (int64_t)gy * W + gx;
        g12[e] = make_float2(2.f * my * (A2 - A1) * iB1 * iB2 - 2.f * mx * ssim * (iB1 - iB2), -ssim * iB2);
        g3[e] = 2.f * A1 * iB1 * iB2;
        const float2 xy = sxy[r0 + o + kHalf][c + kHalf];
        l1 += fabsf(xy.x - xy.y);
        ss += ssim;
    }
    l1 = warp_sum(l1);
    ss = warp_sum(ss);
    if ((t & 31) == 0) {
        red[0][t >> 5] = l1;
        red[1][t >> 5] = ss;
    }
    __syncthreads();
    if (t == 0) {
        double a = 0.0, b = 0.0;
#pragma unroll
        for (int w = 0; w < kLossThreads / 32; w++) {
            a += red[0][w];
            b += red[1][w];
        }
        const int64_t blk = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
        partial[2 * blk] = a;
        partial[2 * blk + 1] = b;
    }
}

// L = scale ((1 - lambda) sum |x - y| + lambda (n_elem - sum SSIM)) from the
// per-block sums of pass 1, in a fixed order; one block, all threads.
__device__ __forceinline__ void loss_total(const double *__restrict__ partial, int64_t blocks, double n_elem,
                                           double lambda, double scale, double *__restrict__ loss, int accumulate)
{
    __shared__ double red[2][kLossThreads];
    double a = 0.0, b = 0.0;
    for (int64_t i = threadIdx.x; i < blocks; i += kLossThreads) {
        a += partial[2 * i];
        b += partial[2 * i + 1];
    }
    red[0][threadIdx.x] = a;
    red[1][threadIdx.x] = b;
    __syncthreads();
    for (int off = kLossThreads / 2; off > 0; off >>= 1) {
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

__global__ void __launch_bounds__(kLossThreads) k_ssim_bwd(const float *__restrict__ x, const float *__restrict__ y,
                                                          int H, int W, const float2 *__restrict__ g12,
                                                          const float *__restrict__ g3, float lambda, float scale,
                                                          float *__restrict__ dx, const double *__restrict__ partial,
                                                          double n_elem, double scale_d, double *__restrict__ loss,
                                                          int accumulate)
{
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0)   // block-uniform
        loss_total(partial, (int64_t)gridDim.x * gridDim.y * gridDim.z, n_elem, (double)lambda, scale_d, loss,
                   accumulate);
    __shared__ __align__(16) float2 s12[kSH][kSWP];   // (g1, g2) with halo
    __shared__ float s3[kSH][kSWP];                   // g3 with halo
    __shared__ __align__(16) float2 h12[kSH][kHP];
    __shared__ float h3[kSH][kHP];
    const int plane = blockIdx.z;
    const int ox = blockIdx.x * kTW, oy = blockIdx.y * kTH;
    const int64_t base = (int64_t)plane * H * W;
    const float2 *p12 = g12 + base;
    const float *p3 = g3 + base;
    stage_tile(s12, ox, oy, H, W, [&](bool in, int64_t e) { return in ? p12[e] : make_float2(0.f, 0.f); });
    stage_tile(s3, ox, oy, H, W, [&](bool in, int64_t e) { return in ? p3[e] : 0.f; });
    __syncthreads();
    const int t = threadIdx.x;
    if (t < kSH * kSegs) {
        const int r = t / kSegs, c0 = (t - r * kSegs) * kSeg;
        float2 a[kSeg + kWin - 1];
        float b[kSeg + kWin - 1];
#pragma unroll
        for (int j = 0; j < kSeg + kWin - 1; j++) {
            a[j] = s12[r][c0 + j];
            b[j] = s3[r][c0 + j];
        }
#pragma unroll
        for (int o = 0; o < kSeg; o++) {
            float2 m = make_float2(0.f, 0.f);
            float d = 0.f;
#pragma unroll
            for (int k = 0; k < kWin; k++) {
                const float w = c_win[k];
                m = __ffma2_rn(f2(w), a[o + k], m);
                d = fmaf(w, b[o + k], d);
            }
            if (c0 + o < kTW) {
                h12[r][c0 + o] = m;
                h3[r][c0 + o] = d;
            }
        }
    }
    __syncthreads();
    const int c = t & 31, r0 = (t >> 5) * kVRows;
    float2 a_in[kVRows + kWin - 1];
    float b_in[kVRows + kWin - 1];
#pragma unroll
    for (int j = 0; j < kVRows + kWin - 1; j++) {
        a_in[j] = h12[r0 + j][c];
        b_in[j] = h3[r0 + j][c];
    }
    const int gx = ox + c;
    float xs[kVRows], ys[kVRows];
#pragma unroll
    for (int o = 0; o < kVRows; o++) {     // issue the pixel loads first
        const int gy = oy + r0 + o;
        const bool in = gy < H && gx < W;
        const int64_t e = base + (int64_t)gy * W + gx;
        xs[o] = in ? x[e] : 0.f;
        ys[o] = in ? y[e] : 0.f;
    }
#pragma unroll
    for (int o = 0; o < kVRows; o++) {
        float2 m = make_float2(0.f, 0.f);
        float d = 0.f;
#pragma unroll
        for (int k = 0; k < kWin; k++) {
            const float w = c_win[k];
            m = __ffma2_rn(f2(w), a_in[o + k], m);
            d = fmaf(w, b_in[o + k], d);
        }
        const int gy = oy + r0 + o;
        if (gy >= H || gx >= W) continue;
        const int64_t e = base + (int64_t)gy * W + gx;
        const float xv = xs[o], yv = ys[o];
        const float diff = xv - yv;
        const float sgn = diff > 0.f ? 1.f : (diff < 0.f ? -1.f : 0.f);
        const float dssim = m.x + 2.f * xv * m.y + yv * d;
        dx[e] = scale * ((1.f - lambda) * sgn - lambda * dssim);
    }
}

// The window lives in __constant__ memory, which each device holds separately:
// the upload is tracked per device (the first loss call on a device makes it).
constexpr int kMaxWinDevices = 64;
std::mutex g_win_mutex;
bool g_win_ready[kMaxWinDevices] = {};

vbm_status ensure_window()
{
    int dev = 0;
    VBM_CUDA(cudaGetDevice(&dev));
    VBM_ARG(dev >= 0 && dev < kMaxWinDevices, "device index out of range");
    std::lock_guard<std::mutex> lock(g_win_mutex);
    if (g_win_ready[dev]) return VBM_OK;
    double g[kWin], s = 0.0;
    for (int i = 0; i < kWin; i++) {
        const double d = i - kHalf;
        g[i] = std::exp(-d * d / (2.0 * 1.5 * 1.5));
        s += g[i];
    }
    float w[kWin];
    for (int i = 0; i < kWin; i++) w[i] = (float)(g[i] / s);
    VBM_CUDA(cudaMemcpyToSymbol(c_win, w, sizeof(w)));
    g_win_ready[dev] = true;
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

int loss_max_images()
{
    return 65535 / 3;     // one grid z-slice per (image, channel)
}

vbm_status loss_fwd_bwd(const float *img, const float *target, int n_images, int H, int W, float lambda,
                        double scale, double *loss, int accumulate, float *dimg, void *ws, cudaStream_t st)
{
    VBM_ARG(n_images <= loss_max_images(), "loss batch of more than 21845 images (3 channels each exceed the "
                                           "grid's 65535 z-slices): split it and use accumulate");
    vbm_status s = ensure_window();
    if (s != VBM_OK) return s;
    const size_t n = (size_t)n_images * 3 * H * W;
    char *p = (char *)ws;
    float2 *g12 = (float2 *)p;
    float *g3 = (float *)(g12 + n);
    size_t off = (3 * n * sizeof(float) + 255) / 256 * 256;
    double *partial = (double *)(p + off);
    dim3 grid((W + kTW - 1) / kTW, (H + kTH - 1) / kTH, n_images * 3);
    k_ssim_fwd<<<grid, kLossThreads, 0, st>>>(img, target, H, W, g12, g3, partial);
    VBM_LAUNCH("ssim_fwd");
    k_ssim_bwd<<<grid, kLossThreads, 0, st>>>(img, target, H, W, g12, g3, lambda, (float)scale, dimg, partial,
                                              (double)n, scale, loss, accumulate);
    VBM_LAUNCH("ssim_bwd");
    note_launches(2);
    return VBM_OK;
}

}  // namespace vbm
