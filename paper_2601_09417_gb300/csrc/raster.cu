// Front-to-back alpha compositing of the binned splats and its reverse-order
// backward (Sec. 4.4, "as in" 3D Gaussian Splatting).
//
// One block per image tile, one thread per pixel.  A tile's depth-ordered
// list is staged through shared memory NT entries at a time: each thread
// gathers one entry's splat record (two float4 and a float) so every pixel of
// the tile reads it from shared memory.  The conic is pre-scaled by
// -log2(e)/2 at staging, so the exponent is evaluated in base 2 with one
// ex2.approx instruction (relative error ~2^-22) per (pixel, Gaussian) pair.
// Early termination: a pixel stops once its transmittance would fall below
// 1e-4, and the whole block leaves the list as soon as __syncthreads_count
// reports every pixel done.
//
// The backward walks each tile's list from the back, starting at the largest
// contributor count of the block, recovers the transmittance by division and
// accumulates per-(view, Gaussian) gradients.  Per pair, the nine partials of
// a warp are summed with shuffles before one atomicAdd per value, and warps
// with no contributing pixel skip the reduction (warp ballot).
#include "vbm_internal.h"

namespace vbm {
namespace {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;
constexpr float kHalfLog2e = -0.5f * kLog2e;   // scales A and C
constexpr float kNegLog2e = -kLog2e;           // scales B

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Base-2 exponent of a staged splat at a pixel, p2 = A' dx^2 + C' dy^2 +
// B' dx dy, with an explicit rounding sequence so the backward recomputes
// exactly the forward's alpha (and therefore the same skip decisions).
struct SplatEval {
    float dx, dy, p2, G, raw;
};

__device__ __forceinline__ SplatEval splat_eval(const float4 g, const float cc, const float opac, const float pxc,
                                                const float pyc)
{
    SplatEval e;
    e.dx = __fsub_rn(g.x, pxc);
    e.dy = __fsub_rn(g.y, pyc);
    float t = __fmul_rn(__fmul_rn(g.z, e.dx), e.dx);
    t = __fmaf_rn(__fmul_rn(cc, e.dy), e.dy, t);
    e.p2 = __fmaf_rn(__fmul_rn(g.w, e.dx), e.dy, t);
    e.G = ex2_approx(e.p2);
    e.raw = __fmul_rn(opac, e.G);
    return e;
}

template <int NT>
__global__ void __launch_bounds__(NT) k_raster_fwd(const int2 *__restrict__ ranges,
                                                   const uint32_t *__restrict__ pair_item,
                                                   const float4 *__restrict__ geo, const float4 *__restrict__ col,
                                                   const float *__restrict__ conic_c, int W, int H, int tw, int TX,
                                                   int TY, int vb, float bg0, float bg1, float bg2,
                                                   float *__restrict__ img, float *__restrict__ alpha_out,
                                                   float *__restrict__ T_final, int32_t *__restrict__ n_contrib,
                                                   int32_t *__restrict__ n_eval)
{
    __shared__ float4 s_geo[NT];   // u, v, A', B'
    __shared__ float4 s_col[NT];   // r, g, b, opacity
    __shared__ float s_c[NT];      // C'
    const int tiles_per_view = TX * TY;
    const int vrel = blockIdx.x / tiles_per_view;
    const int t = blockIdx.x - vrel * tiles_per_view;
    const int ty = t / TX, tx = t - ty * TX;
    const int th = NT / tw;
    const int px = tx * tw + (int)(threadIdx.x % tw);
    const int py = ty * th + (int)(threadIdx.x / tw);
    const bool inside = px < W && py < H;
    const float pxc = px + 0.5f, pyc = py + 0.5f;
    const int2 rg = ranges[blockIdx.x];
    bool done = !inside;
    float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f;
    int last = 0;
    int evaluated = rg.y - rg.x;
    for (int base = rg.x; base < rg.y; base += NT) {
        if (__syncthreads_count(done) == NT) break;
        const int idx = base + threadIdx.x;
        if (idx < rg.y) {
            const uint32_t it = pair_item[idx];
            const float4 g = geo[it];
            s_geo[threadIdx.x] = make_float4(g.x, g.y, g.z * kHalfLog2e, g.w * kNegLog2e);
            s_c[threadIdx.x] = conic_c[it] * kHalfLog2e;
            s_col[threadIdx.x] = col[it];
        }
        __syncthreads();
        const int n = min(NT, rg.y - base);
        if (!done) {
            for (int j = 0; j < n; j++) {
                const float4 c = s_col[j];
                const SplatEval e = splat_eval(s_geo[j], s_c[j], c.w, pxc, pyc);
                if (e.p2 > 0.f) continue;
                const float alpha = fminf(kAlphaMax, e.raw);
                if (alpha < kAlphaMin) continue;
                const float testT = T * (1.f - alpha);
                if (testT < kTMin) {
                    done = true;
                    evaluated = base - rg.x + j + 1;
                    break;
                }
                const float wgt = alpha * T;
                C0 += c.x * wgt;
                C1 += c.y * wgt;
                C2 += c.z * wgt;
                T = testT;
                last = base - rg.x + j + 1;
            }
        }
    }
    if (inside) {
        const int64_t HW = (int64_t)H * W;
        const int64_t v = vb + vrel;
        const int64_t pix = (int64_t)py * W + px;
        img[(v * 3 + 0) * HW + pix] = C0 + T * bg0;
        img[(v * 3 + 1) * HW + pix] = C1 + T * bg1;
        img[(v * 3 + 2) * HW + pix] = C2 + T * bg2;
        if (alpha_out) alpha_out[v * HW + pix] = 1.f - T;
        T_final[v * HW + pix] = T;
        n_contrib[v * HW + pix] = last;
        if (n_eval) n_eval[v * HW + pix] = evaluated;
    }
}

__device__ __forceinline__ float warp_sum(float x)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    return x;
}

template <int NT>
__global__ void __launch_bounds__(NT) k_raster_bwd(const int2 *__restrict__ ranges,
                                                   const uint32_t *__restrict__ pair_item,
                                                   const float4 *__restrict__ geo, const float4 *__restrict__ col,
                                                   const float *__restrict__ conic_c, int W, int H, int tw, int TX,
                                                   int TY, int vb, float bg0, float bg1, float bg2,
                                                   const float *__restrict__ dimg, const float *__restrict__ dalpha,
                                                   const float *__restrict__ T_final,
                                                   const int32_t *__restrict__ n_contrib, float *__restrict__ gs,
                                                   int64_t n_items)
{
    __shared__ float4 s_geo[NT];
    __shared__ float4 s_col[NT];
    __shared__ float s_c[NT];
    __shared__ uint32_t s_item[NT];
    __shared__ int s_max;
    const int tiles_per_view = TX * TY;
    const int vrel = blockIdx.x / tiles_per_view;
    const int t = blockIdx.x - vrel * tiles_per_view;
    const int ty = t / TX, tx = t - ty * TX;
    const int th = NT / tw;
    const int px = tx * tw + (int)(threadIdx.x % tw);
    const int py = ty * th + (int)(threadIdx.x / tw);
    const bool inside = px < W && py < H;
    const float pxc = px + 0.5f, pyc = py + 0.5f;
    const int2 rg = ranges[blockIdx.x];
    const int64_t HW = (int64_t)H * W;
    const int64_t v = vb + vrel;
    const int64_t pix = (int64_t)py * W + px;
    float T = 1.f, dC0 = 0.f, dC1 = 0.f, dC2 = 0.f, dA = 0.f;
    int nc = 0;
    if (inside) {
        T = T_final[v * HW + pix];
        nc = n_contrib[v * HW + pix];
        dC0 = dimg[(v * 3 + 0) * HW + pix];
        dC1 = dimg[(v * 3 + 1) * HW + pix];
        dC2 = dimg[(v * 3 + 2) * HW + pix];
        if (dalpha) dA = dalpha[v * HW + pix];
    }
    const float Tf = T;
    // constant part of dL/dalpha_k * (1 - alpha_k): background and alpha-output terms
    const float tail = Tf * (bg0 * dC0 + bg1 * dC1 + bg2 * dC2) - dA * Tf;
    float S0 = 0.f, S1 = 0.f, S2 = 0.f;   // sum over later contributors of c alpha T
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    atomicMax(&s_max, nc);
    __syncthreads();
    const int max_nc = s_max;
    const int lane = threadIdx.x & 31;
    for (int hi = max_nc; hi > 0; hi -= NT) {
        const int lo = max(0, hi - NT);
        __syncthreads();
        const int pos_load = lo + (int)threadIdx.x;
        if (pos_load < hi) {
            const uint32_t it = pair_item[rg.x + pos_load];
            const float4 g = geo[it];
            s_geo[threadIdx.x] = make_float4(g.x, g.y, g.z * kHalfLog2e, g.w * kNegLog2e);
            s_c[threadIdx.x] = conic_c[it] * kHalfLog2e;
            s_col[threadIdx.x] = col[it];
            s_item[threadIdx.x] = it;
        }
        __syncthreads();
        for (int j = hi - 1 - lo; j >= 0; j--) {
            const int pos = lo + j;
            float g_u = 0.f, g_v = 0.f, g_a = 0.f, g_b = 0.f, g_c = 0.f, g_o = 0.f, g_r = 0.f, g_g = 0.f,
                  g_bl = 0.f;
            bool contrib = false;
            if (pos < nc) {
                const float4 g = s_geo[j];
                const float cc = s_c[j];
                const float4 c = s_col[j];
                const SplatEval e = splat_eval(g, cc, c.w, pxc, pyc);
                const float dx = e.dx, dy = e.dy, G = e.G, raw = e.raw;
                const float alpha = fminf(kAlphaMax, raw);
                if (e.p2 <= 0.f && alpha >= kAlphaMin) {
                    contrib = true;
                    const float om = 1.f - alpha;
                    T = T / om;
                    const float wgt = alpha * T;
                    g_r = wgt * dC0;
                    g_g = wgt * dC1;
                    g_bl = wgt * dC2;
                    const float dLda = (c.x * T * dC0 + c.y * T * dC1 + c.z * T * dC2) -
                                       (S0 * dC0 + S1 * dC1 + S2 * dC2 + tail) / om;
                    S0 += c.x * wgt;
                    S1 += c.y * wgt;
                    S2 += c.z * wgt;
                    if (raw < kAlphaMax) {
                        const float dpow = dLda * raw;   // dL/dpower = dL/dalpha * o * G
                        g_o = dLda * G;
                        // natural-log exponent derivatives; A' = -log2e A / 2, B' = -log2e B
                        g_u = dpow * kLn2 * (2.f * g.z * dx + g.w * dy);
                        g_v = dpow * kLn2 * (2.f * cc * dy + g.w * dx);
                        g_a = dpow * (-0.5f * dx * dx);
                        g_b = dpow * (-dx * dy);
                        g_c = dpow * (-0.5f * dy * dy);
                    }
                }
            }
            if (__any_sync(0xffffffffu, contrib)) {
                g_u = warp_sum(g_u);
                g_v = warp_sum(g_v);
                g_a = warp_sum(g_a);
                g_b = warp_sum(g_b);
                g_c = warp_sum(g_c);
                g_o = warp_sum(g_o);
                g_r = warp_sum(g_r);
                g_g = warp_sum(g_g);
                g_bl = warp_sum(g_bl);
                if (lane == 0) {
                    const uint32_t it = s_item[j];
                    atomicAdd(&gs[0 * n_items + it], g_u);
                    atomicAdd(&gs[1 * n_items + it], g_v);
                    atomicAdd(&gs[2 * n_items + it], g_a);
                    atomicAdd(&gs[3 * n_items + it], g_b);
                    atomicAdd(&gs[4 * n_items + it], g_c);
                    atomicAdd(&gs[5 * n_items + it], g_o);
                    atomicAdd(&gs[6 * n_items + it], g_r);
                    atomicAdd(&gs[7 * n_items + it], g_g);
                    atomicAdd(&gs[8 * n_items + it], g_bl);
                }
            }
        }
    }
}

template <int NT>
vbm_status launch_fwd(vbm_plan *p, int vb, int vc, const float bg[3], float *img, float *alpha, cudaStream_t st)
{
    const int blocks = vc * p->TX * p->TY;
    record_event(p->prof_ev[0], st);
    k_raster_fwd<NT><<<blocks, NT, 0, st>>>(p->ranges, p->pair_item[p->pair_buf], p->geo, p->col, p->conic_c,
                                             p->desc.width, p->desc.height, p->desc.tile_w, p->TX, p->TY, vb, bg[0],
                                             bg[1], bg[2], img, alpha, p->T_final, p->n_contrib, p->prof_n_eval);
    VBM_LAUNCH("raster_fwd");
    record_event(p->prof_ev[1], st);
    note_launches(1);
    return VBM_OK;
}

template <int NT>
vbm_status launch_bwd(vbm_plan *p, int vb, int vc, const float bg[3], const float *dimg, const float *dalpha,
                      cudaStream_t st)
{
    const int blocks = vc * p->TX * p->TY;
    record_event(p->prof_ev[2], st);
    k_raster_bwd<NT><<<blocks, NT, 0, st>>>(p->ranges, p->pair_item[p->pair_buf], p->geo, p->col, p->conic_c,
                                             p->desc.width, p->desc.height, p->desc.tile_w, p->TX, p->TY, vb, bg[0],
                                             bg[1], bg[2], dimg, dalpha, p->T_final, p->n_contrib, p->g_splat,
                                             p->last_items);
    VBM_LAUNCH("raster_bwd");
    record_event(p->prof_ev[3], st);
    note_launches(1);
    return VBM_OK;
}

}  // namespace

vbm_status raster_fwd(vbm_plan *p, int vb, int vc, const float bg[3], float *img, float *alpha, cudaStream_t st)
{
    switch (p->desc.tile_w * p->desc.tile_h) {
        case 64: return launch_fwd<64>(p, vb, vc, bg, img, alpha, st);
        case 128: return launch_fwd<128>(p, vb, vc, bg, img, alpha, st);
        case 256: return launch_fwd<256>(p, vb, vc, bg, img, alpha, st);
        default: set_error("tile_w * tile_h must be 64, 128 or 256"); return VBM_ERR_ARG;
    }
}

vbm_status raster_bwd(vbm_plan *p, const float *, int64_t, int vb, int vc, const float bg[3], const float *dimg,
                      const float *dalpha, float *, cudaStream_t st)
{
    VBM_CUDA(cudaMemsetAsync(p->g_splat, 0, sizeof(float) * 9 * p->last_items, st));
    switch (p->desc.tile_w * p->desc.tile_h) {
        case 64: return launch_bwd<64>(p, vb, vc, bg, dimg, dalpha, st);
        case 128: return launch_bwd<128>(p, vb, vc, bg, dimg, dalpha, st);
        case 256: return launch_bwd<256>(p, vb, vc, bg, dimg, dalpha, st);
        default: set_error("tile_w * tile_h must be 64, 128 or 256"); return VBM_ERR_ARG;
    }
}

}  // namespace vbm
