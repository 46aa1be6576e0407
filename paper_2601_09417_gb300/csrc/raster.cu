// Front-to-back alpha compositing of the binned splats and its reverse-order
// backward (Sec. 4.4, "as in" 3D Gaussian Splatting).
//
// One block per image tile.  Each thread owns PPT consecutive pixels of one
// tile column, so the per-splat work that only depends on the column
// (shared-memory loads, dx, A' dx^2, B' dx) is done once per thread, the
// per-pixel arithmetic of two pixels is issued as packed FP32x2 operations
// (__ffma2_rn / __fmul2_rn / __fadd2_rn, sm_100+), and each warp covers a
// compact rectangle of the tile.
//
// A tile's depth-ordered list is staged through shared memory NT entries at a
// time.  While staging, each entry is tested against the tile: the minimum of
// its quadratic form over the rectangle of the tile's pixel centres gives the
// largest alpha any pixel of the tile can see; entries below the 1/255
// cut-off (with a 1e-3 margin in the exponent, far above rounding) are
// dropped and the rest compacted in list order.  A dropped entry would have
// been skipped by every pixel, so the image, the saved state and the
// gradients are unchanged; the original list position travels with each
// entry for the contributor count.  Each staged entry also carries the
// bounding box of its alpha >= 1/255 ellipse; a warp whose pixel rectangle
// misses that box skips the entry with one warp-uniform test (no pixel of
// the warp could composite it).
//
// The conic is pre-scaled by -log2(e)/2 when staged, so the exponent is one
// ex2.approx.ftz per (pixel, splat) pair; its rounding sequence is fixed
// (explicit _rn operations) so the backward recomputes exactly the forward's
// alphas and skip decisions.  A pixel stops once its transmittance would
// fall below 1e-4; the block leaves the list when __syncthreads_count reports
// every pixel done.
//
// The backward walks each tile's list from the back, starting at the largest
// contributor count of the block, recovers the transmittance by division and
// accumulates per-(view, splat) gradients: per splat, the nine partials are
// summed over a warp by a 12-shuffle reduce-scatter (skipped by ballot when
// no lane contributes), over the block through shared memory in groups of 32 splats,
// and then added to global memory with nine atomics per (splat, tile).  A warp
// also skips entries beyond the largest contributor count of its pixels.
#include "vbm_internal.h"

namespace vbm {
namespace {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;
constexpr float kHalfLog2e = -0.5f * kLog2e;   // scales A and C
constexpr float kNegLog2e = -kLog2e;           // scales B
constexpr float kCullMargin = 1e-3f;           // natural-log margin of the tile test

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Smallest q = A dx^2 + 2 B dx dy + C dy^2 (dx = x - u, dy = y - v) over the
// rectangle [x0, x1] x [y0, y1]: 0 inside, else the minimum over the four
// edges, each the clamped 1D minimiser.
__device__ __forceinline__ float rect_min_quadratic(float u, float v, float A, float B, float C, float x0, float x1,
                                                    float y0, float y1)
{
    if (u >= x0 && u <= x1 && v >= y0 && v <= y1) return 0.f;
    float best = 3.4e38f;
#pragma unroll
    for (int e = 0; e < 2; e++) {
        const float dx = (e ? x1 : x0) - u;
        const float dy = fminf(fmaxf(v - B * dx / C, y0), y1) - v;
        best = fminf(best, A * dx * dx + 2.f * B * dx * dy + C * dy * dy);
        const float ey = (e ? y1 : y0) - v;
        const float ex = fminf(fmaxf(u - B * ey / A, x0), x1) - u;
        best = fminf(best, A * ex * ex + 2.f * B * ex * ey + C * ey * ey);
    }
    return best;
}

struct TileGeom {
    int vrel, px, py0;
    float pxc;
    float x0, x1, y0, y1;       // pixel-centre rectangle of the tile (clipped to the image)
    float wx0, wx1, wy0, wy1;   // pixel-centre rectangle of this thread's warp (clipped)
};

template <int NT, int PPT>
__device__ __forceinline__ TileGeom tile_geom(int tile, int tw, int TX, int TY, int W, int H)
{
    constexpr int NPIX = NT * PPT;
    const int th = NPIX / tw;
    TileGeom t;
    const int tiles_per_view = TX * TY;
    t.vrel = tile / tiles_per_view;
    const int tt = tile - t.vrel * tiles_per_view;
    const int ty = tt / TX, tx = tt - ty * TX;
    t.px = tx * tw + (int)(threadIdx.x % tw);
    t.py0 = ty * th + (int)(threadIdx.x / tw) * PPT;
    t.pxc = t.px + 0.5f;
    t.x0 = tx * tw + 0.5f;
    t.x1 = min(tx * tw + tw, W) - 0.5f;
    t.y0 = ty * th + 0.5f;
    t.y1 = min(ty * th + th, H) - 0.5f;
    // a warp holds threads [32 w, 32 w + 32): whole tile rows when tw divides 32
    const int w = threadIdx.x >> 5;
    const int g0 = (32 * w) / tw, g1 = (32 * w + 31) / tw;
    t.wx0 = t.x0;
    t.wx1 = t.x1;
    t.wy0 = ty * th + g0 * PPT + 0.5f;
    t.wy1 = fminf((float)(ty * th + (g1 + 1) * PPT), (float)H) - 0.5f;
    return t;
}

// Stage entries [base, min(base + NT, end)) of a tile list: test each against
// the tile and compact the survivors, in list order, into shared memory.
// Returns the number staged.  All threads of the block must call it.
template <int NT>
__device__ __forceinline__ int stage_entries(int base, int end, int list_begin, const uint32_t *__restrict__ pair_item,
                                             const float4 *__restrict__ geo, const float4 *__restrict__ col,
                                             const float *__restrict__ conic_c, const TileGeom &tg, float4 *s_geo,
                                             float4 *s_col, float2 *s_cp, float4 *s_box, uint32_t *s_item,
                                             int *s_warp)
{
    const int idx = base + (int)threadIdx.x;
    bool keep = false;
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f), c = g, box = g;
    float cc = 0.f;
    uint32_t it = 0;
    if (idx < end) {
        it = pair_item[idx];
        g = geo[it];
        cc = conic_c[it];
        c = col[it];
        const float q = rect_min_quadratic(g.x, g.y, g.z, g.w, cc, tg.x0, tg.x1, tg.y0, tg.y1);
        const float tau = 2.f * (logf(255.f * c.w) + kCullMargin);
        keep = 0.5f * q <= 0.5f * tau;
        // bounding box of {q <= tau}: half-widths sqrt(tau C / det), sqrt(tau A / det) of the conic
        const float det = g.z * cc - g.w * g.w;
        const float hx = sqrtf(fmaxf(tau, 0.f) * cc / det) * 1.0001f + 1e-3f;
        const float hy = sqrtf(fmaxf(tau, 0.f) * g.z / det) * 1.0001f + 1e-3f;
        box = make_float4(g.x - hx, g.x + hx, g.y - hy, g.y + hy);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t bal = __ballot_sync(0xffffffffu, keep);
    __syncthreads();            // the previous batch is no longer read
    if (lane == 0) s_warp[warp] = __popc(bal);
    __syncthreads();
    int before = 0, total = 0;
#pragma unroll
    for (int w = 0; w < NT / 32; w++) {
        const int cnt = s_warp[w];
        before += w < warp ? cnt : 0;
        total += cnt;
    }
    if (keep) {
        const int slot = before + __popc(bal & ((1u << lane) - 1u));
        s_geo[slot] = make_float4(g.x, g.y, g.z * kHalfLog2e, g.w * kNegLog2e);
        s_cp[slot] = make_float2(cc * kHalfLog2e, __int_as_float(idx - list_begin));
        s_col[slot] = c;
        s_box[slot] = box;
        if (s_item) s_item[slot] = it;
    }
    __syncthreads();
    return total;
}

// Per-pixel compositing state of a thread's pixels after the forward walk.
template <int PPT>
struct PixState {
    float T[PPT];
    int last[PPT];
};

// Forward walk of one tile.  COLOR = false computes only the per-pixel state
// (final transmittance and last contributor), with exactly the decisions of
// the full forward: the backward uses it when the state is not stored.
template <int NT, int PPT, bool COLOR = true>
__device__ __forceinline__ void fwd_tile(const int tile, const int2 *__restrict__ ranges,
                                                   const uint32_t *__restrict__ pair_item,
                                                   const float4 *__restrict__ geo, const float4 *__restrict__ col,
                                                   const float *__restrict__ conic_c, int W, int H, int tw, int TX,
                                                   int TY, int vb, float bg0, float bg1, float bg2,
                                                   float *__restrict__ img, float *__restrict__ alpha_out,
                                                   float *__restrict__ T_final, int32_t *__restrict__ n_contrib,
                                                   int32_t *__restrict__ n_eval, PixState<PPT> *state = nullptr)
{
    static_assert(PPT == 1 || PPT % 2 == 0, "pixels per thread: 1 or even");
    constexpr int STEP = PPT == 1 ? 1 : 2;
    __shared__ float4 s_geo[NT];
    __shared__ float4 s_col[NT];
    __shared__ float2 s_cp[NT];
    __shared__ float4 s_box[NT];
    __shared__ int s_warp[NT / 32];
    const TileGeom tg = tile_geom<NT, PPT>(tile, tw, TX, TY, W, H);
    const int2 rg = ranges[tile];
    float pyc[PPT], T[PPT], C0[PPT], C1[PPT], C2[PPT];
    int last[PPT], evaluated[PPT];
    bool inside[PPT], done[PPT];
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        const int py = tg.py0 + k;
        pyc[k] = py + 0.5f;
        inside[k] = tg.px < W && py < H;
        done[k] = !inside[k];
        T[k] = 1.f;
        C0[k] = C1[k] = C2[k] = 0.f;
        last[k] = 0;
        evaluated[k] = rg.y - rg.x;
    }
    for (int base = rg.x; base < rg.y; base += NT) {
        bool all_done = true;
#pragma unroll
        for (int k = 0; k < PPT; k++) all_done &= done[k];
        if (__syncthreads_count(all_done) == NT) break;
        const int n = stage_entries<NT>(base, rg.y, rg.x, pair_item, geo, col, conic_c, tg, s_geo, s_col, s_cp,
                                        s_box, nullptr, s_warp);
        if (all_done) continue;
        for (int j = 0; j < n; j++) {
            const float4 bx = s_box[j];
            if (bx.y < tg.wx0 || bx.x > tg.wx1 || bx.w < tg.wy0 || bx.z > tg.wy1) continue;   // warp-uniform
            const float4 g = s_geo[j];
            const float2 cp = s_cp[j];
            const float4 c = s_col[j];
            const int pos = __float_as_int(cp.y);
            const float dx = __fsub_rn(g.x, tg.pxc);
            const float t0 = __fmul_rn(__fmul_rn(g.z, dx), dx);
            const float bdx = __fmul_rn(g.w, dx);
#pragma unroll
            for (int k = 0; k < PPT; k += STEP) {
                float p2[2], raw[2];
                if (PPT == 1) {
                    const float dy = __fsub_rn(g.y, pyc[k]);
                    const float t = __fmaf_rn(__fmul_rn(cp.x, dy), dy, t0);
                    p2[0] = __fmaf_rn(bdx, dy, t);
                    raw[0] = __fmul_rn(c.w, ex2_approx(p2[0]));
                } else {
                    // a - b == a + (-b) exactly, so this matches __fsub_rn in the backward
                    const float2 dy = __fadd2_rn(make_float2(g.y, g.y), make_float2(-pyc[k], -pyc[k + STEP - 1]));
                    const float2 t = __ffma2_rn(__fmul2_rn(make_float2(cp.x, cp.x), dy), dy, make_float2(t0, t0));
                    const float2 q = __ffma2_rn(make_float2(bdx, bdx), dy, t);
                    p2[0] = q.x;
                    p2[1] = q.y;
                    const float2 r = __fmul2_rn(make_float2(c.w, c.w), make_float2(ex2_approx(q.x), ex2_approx(q.y)));
                    raw[0] = r.x;
                    raw[1] = r.y;
                }
#pragma unroll
                for (int h = 0; h < STEP; h++) {
                    const int kk = k + h;
                    const float alpha = fminf(kAlphaMax, raw[h]);
                    const bool cand = !done[kk] && p2[h] <= 0.f && alpha >= kAlphaMin;
                    const float testT = T[kk] * (1.f - alpha);
                    const bool term = cand && testT < kTMin;
                    const bool blend = cand && !term;
                    if (term) {
                        done[kk] = true;
                        evaluated[kk] = pos + 1;
                    }
                    if (COLOR) {
                        const float wgt = blend ? alpha * T[kk] : 0.f;
                        C0[kk] = __fmaf_rn(c.x, wgt, C0[kk]);
                        C1[kk] = __fmaf_rn(c.y, wgt, C1[kk]);
                        C2[kk] = __fmaf_rn(c.z, wgt, C2[kk]);
                    }
                    T[kk] = blend ? testT : T[kk];
                    last[kk] = blend ? pos + 1 : last[kk];
                }
            }
        }
    }
    if (state) {
#pragma unroll
        for (int k = 0; k < PPT; k++) {
            state->T[k] = T[k];
            state->last[k] = last[k];
        }
    }
    if (!COLOR) return;
    const int64_t HW = (int64_t)H * W;
    const int64_t v = vb + tg.vrel;
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        if (!inside[k]) continue;
        const int64_t pix = (int64_t)(tg.py0 + k) * W + tg.px;
        img[(v * 3 + 0) * HW + pix] = C0[k] + T[k] * bg0;
        img[(v * 3 + 1) * HW + pix] = C1[k] + T[k] * bg1;
        img[(v * 3 + 2) * HW + pix] = C2[k] + T[k] * bg2;
        if (alpha_out) alpha_out[v * HW + pix] = 1.f - T[k];
        if (T_final) T_final[v * HW + pix] = T[k];
        if (n_contrib) n_contrib[v * HW + pix] = last[k];
        if (n_eval) n_eval[v * HW + pix] = evaluated[k];
    }
}

// One reduce-scatter step across lanes l and l ^ (1 << bit): for each pair
// (a, b) of the lane's partial sums, the lane keeps a (lower half) or b (upper
// half) and adds the partner's copy of the same element.
template <int NP>
__device__ __forceinline__ void rs_step(const float (&in)[2 * NP], float (&out)[NP], int bit)
{
    const bool hi = (threadIdx.x >> bit) & 1;
#pragma unroll
    for (int i = 0; i < NP; i++) {
        const float a = in[i], b = in[NP + i];
        const float send = hi ? a : b;
        const float keep = hi ? b : a;
        out[i] = keep + __shfl_xor_sync(0xffffffffu, send, 1 << bit);
    }
}

// Sums nine values over the 32 lanes of a warp with 12 shuffles (instead of
// 45 for nine butterfly reductions).  Returns the sum of value
// kRsIndex[lane >> 1] (lanes with an odd index hold the same sum as their
// even neighbour); entries 15 of the table mark lanes that hold no value.
constexpr uint64_t kRsIndex = 0xFFF8F765FF43F210ull;   // nibble m = value held by lanes 2m, 2m+1

__device__ __forceinline__ int rs_value_index(int lane) { return (int)((kRsIndex >> (4 * (lane >> 1))) & 15); }

__device__ __forceinline__ float reduce_scatter9(const float (&v)[9])
{
    const float a[10] = {v[0], v[1], v[2], v[3], v[4], v[5], v[6], v[7], v[8], 0.f};
    float b[5];
    rs_step<5>(a, b, 4);                       // pairs (0,5) (1,6) (2,7) (3,8) (4,-)
    const float b6[6] = {b[0], b[1], b[2], b[3], b[4], 0.f};
    float c[3];
    rs_step<3>(b6, c, 3);                      // pairs (0,3) (1,4) (2,-)
    const float c4[4] = {c[0], c[1], c[2], 0.f};
    float d[2];
    rs_step<2>(c4, d, 2);                      // pairs (0,2) (1,-)
    float e[1];
    rs_step<1>(d, e, 1);                       // pair (0,1)
    return e[0] + __shfl_xor_sync(0xffffffffu, e[0], 1);
}

constexpr int kGroup = 32;   // splats per block-level gradient reduction

template <int NT, int PPT>
__device__ __forceinline__ void bwd_tile(const int tile, const int2 *__restrict__ ranges,
                                                   const uint32_t *__restrict__ pair_item,
                                                   const float4 *__restrict__ geo, const float4 *__restrict__ col,
                                                   const float *__restrict__ conic_c, int W, int H, int tw, int TX,
                                                   int TY, int vb, float bg0, float bg1, float bg2,
                                                   const float *__restrict__ dimg, const float *__restrict__ dalpha,
                                                   const float *__restrict__ T_final,
                                                   const int32_t *__restrict__ n_contrib, float *__restrict__ gs,
                                                   int64_t n_items)
{
    constexpr int NW = NT / 32;
    __shared__ float4 s_geo[NT];
    __shared__ float4 s_col[NT];
    __shared__ float2 s_cp[NT];
    __shared__ float4 s_box[NT];
    __shared__ uint32_t s_item[NT];
    __shared__ int s_warp[NW];
    __shared__ float s_red[NW][kGroup][9];
    __shared__ int s_max;
    const TileGeom tg = tile_geom<NT, PPT>(tile, tw, TX, TY, W, H);
    const int2 rg = ranges[tile];
    const int64_t HW = (int64_t)H * W;
    const int64_t v = vb + tg.vrel;
    float pyc[PPT], T[PPT], dC0[PPT], dC1[PPT], dC2[PPT], tail[PPT], S0[PPT], S1[PPT], S2[PPT];
    int nc[PPT];
    int my_max = 0;
    PixState<PPT> rec;
    if (!T_final) {   // recompute mode: replay the forward decisions of this tile
        fwd_tile<NT, PPT, false>(tile, ranges, pair_item, geo, col, conic_c, W, H, tw, TX, TY, vb, bg0, bg1, bg2,
                                 nullptr, nullptr, nullptr, nullptr, nullptr, &rec);
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        const int py = tg.py0 + k;
        pyc[k] = py + 0.5f;
        T[k] = 1.f;
        dC0[k] = dC1[k] = dC2[k] = 0.f;
        nc[k] = 0;
        float dA = 0.f;
        if (tg.px < W && py < H) {
            const int64_t pix = (int64_t)py * W + tg.px;
            T[k] = T_final ? T_final[v * HW + pix] : rec.T[k];
            nc[k] = T_final ? n_contrib[v * HW + pix] : rec.last[k];
            dC0[k] = dimg[(v * 3 + 0) * HW + pix];
            dC1[k] = dimg[(v * 3 + 1) * HW + pix];
            dC2[k] = dimg[(v * 3 + 2) * HW + pix];
            if (dalpha) dA = dalpha[v * HW + pix];
        }
        // constant part of dL/dalpha_k (1 - alpha_k): background and alpha-output terms
        tail[k] = T[k] * (bg0 * dC0[k] + bg1 * dC1[k] + bg2 * dC2[k]) - dA * T[k];
        S0[k] = S1[k] = S2[k] = 0.f;
        my_max = max(my_max, nc[k]);
    }
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    atomicMax(&s_max, my_max);
    __syncthreads();
    const int max_nc = s_max;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int warp_max_nc = __reduce_max_sync(0xffffffffu, my_max);
    for (int hi = max_nc; hi > 0; hi -= NT) {
        const int lo = max(0, hi - NT);
        const int n = stage_entries<NT>(rg.x + lo, rg.x + hi, rg.x, pair_item, geo, col, conic_c, tg, s_geo, s_col,
                                        s_cp, s_box, s_item, s_warp);
        // walk the compacted batch backwards in groups of kGroup splats
        for (int g_hi = n; g_hi > 0; g_hi -= kGroup) {
            const int g_lo = max(0, g_hi - kGroup);
            for (int j = g_hi - 1; j >= g_lo; j--) {
                const int slot = j - g_lo;
                const float2 cp = s_cp[j];
                const int pos = __float_as_int(cp.y);
                const float4 bx = s_box[j];
                // warp-uniform: no pixel of this warp contributed this entry
                if (pos >= warp_max_nc || bx.y < tg.wx0 || bx.x > tg.wx1 || bx.w < tg.wy0 || bx.z > tg.wy1) {
                    const int vi = rs_value_index(lane);
                    if (!(lane & 1) && vi < 9) s_red[warp][slot][vi] = 0.f;
                    continue;
                }
                const float4 g = s_geo[j];
                const float4 c = s_col[j];
                const float dx = __fsub_rn(g.x, tg.pxc);
                const float t0 = __fmul_rn(__fmul_rn(g.z, dx), dx);
                const float bdx = __fmul_rn(g.w, dx);
                float acc[9];
#pragma unroll
                for (int q = 0; q < 9; q++) acc[q] = 0.f;
                bool any = false;
#pragma unroll
                for (int k = 0; k < PPT; k++) {
                    if (pos >= nc[k]) continue;
                    const float dy = __fsub_rn(g.y, pyc[k]);
                    const float t = __fmaf_rn(__fmul_rn(cp.x, dy), dy, t0);
                    const float p2 = __fmaf_rn(bdx, dy, t);
                    const float G = ex2_approx(p2);
                    const float raw = __fmul_rn(c.w, G);
                    const float alpha = fminf(kAlphaMax, raw);
                    if (p2 <= 0.f && alpha >= kAlphaMin) {
                        any = true;
                        const float r_om = __frcp_rn(1.f - alpha);
                        T[k] = T[k] * r_om;
                        const float wgt = alpha * T[k];
                        acc[6] += wgt * dC0[k];
                        acc[7] += wgt * dC1[k];
                        acc[8] += wgt * dC2[k];
                        const float dLda = (c.x * dC0[k] + c.y * dC1[k] + c.z * dC2[k]) * T[k] -
                                           (S0[k] * dC0[k] + S1[k] * dC1[k] + S2[k] * dC2[k] + tail[k]) * r_om;
                        S0[k] += c.x * wgt;
                        S1[k] += c.y * wgt;
                        S2[k] += c.z * wgt;
                        if (raw < kAlphaMax) {
                            const float dpow = dLda * raw;   // dL/dpower = dL/dalpha o G
                            acc[5] += dLda * G;
                            // natural-log exponent: A' = -log2e A / 2, B' = -log2e B
                            acc[0] += dpow * kLn2 * (2.f * g.z * dx + g.w * dy);
                            acc[1] += dpow * kLn2 * (2.f * cp.x * dy + g.w * dx);
                            acc[2] += dpow * (-0.5f * dx * dx);
                            acc[3] += dpow * (-dx * dy);
                            acc[4] += dpow * (-0.5f * dy * dy);
                        }
                    }
                }
                const int vi = rs_value_index(lane);
                const float sum = __any_sync(0xffffffffu, any) ? reduce_scatter9(acc) : 0.f;
                if (!(lane & 1) && vi < 9) s_red[warp][slot][vi] = sum;
            }
            __syncthreads();
            const int cnt = g_hi - g_lo;
            for (int e = threadIdx.x; e < cnt * 9; e += NT) {
                const int slot = e / 9, q = e - slot * 9;
                float sum = 0.f;
#pragma unroll
                for (int w = 0; w < NW; w++) sum += s_red[w][slot][q];
                if (sum != 0.f) atomicAdd(&gs[(int64_t)q * n_items + s_item[g_lo + slot]], sum);
            }
            __syncthreads();
        }
    }
}

// Kernels: one block per tile, or (PERSIST) a grid of SMs x resident blocks
// whose blocks take tiles from an atomic queue in longest-list-first order.
template <int NT, int PPT, bool PERSIST>
__global__ void __launch_bounds__(NT) k_raster_fwd(const int *__restrict__ order, int *__restrict__ queue,
                                                   int n_tiles, const int2 *__restrict__ ranges, const uint32_t *__restrict__ pair_item, const float4 *__restrict__ geo, const float4 *__restrict__ col, const float *__restrict__ conic_c, int W, int H, int tw, int TX, int TY, int vb, float bg0, float bg1, float bg2, float *__restrict__ img, float *__restrict__ alpha_out, float *__restrict__ T_final, int32_t *__restrict__ n_contrib, int32_t *__restrict__ n_eval)
{
    if constexpr (!PERSIST) {
        fwd_tile<NT, PPT>(blockIdx.x, ranges, pair_item, geo, col, conic_c, W, H, tw, TX, TY, vb, bg0, bg1, bg2, img, alpha_out, T_final, n_contrib, n_eval);
    } else {
        __shared__ int s_next;
        for (;;) {
            __syncthreads();
            if (threadIdx.x == 0) s_next = atomicAdd(queue, 1);
            __syncthreads();
            const int q = s_next;
            if (q >= n_tiles) return;
            fwd_tile<NT, PPT>(order[q], ranges, pair_item, geo, col, conic_c, W, H, tw, TX, TY, vb, bg0, bg1, bg2, img, alpha_out, T_final, n_contrib, n_eval);
        }
    }
}

template <int NT, int PPT, bool PERSIST>
__global__ void __launch_bounds__(NT) k_raster_bwd(const int *__restrict__ order, int *__restrict__ queue,
                                                   int n_tiles, const int2 *__restrict__ ranges, const uint32_t *__restrict__ pair_item, const float4 *__restrict__ geo, const float4 *__restrict__ col, const float *__restrict__ conic_c, int W, int H, int tw, int TX, int TY, int vb, float bg0, float bg1, float bg2, const float *__restrict__ dimg, const float *__restrict__ dalpha, const float *__restrict__ T_final, const int32_t *__restrict__ n_contrib, float *__restrict__ gs, int64_t n_items)
{
    if constexpr (!PERSIST) {
        bwd_tile<NT, PPT>(blockIdx.x, ranges, pair_item, geo, col, conic_c, W, H, tw, TX, TY, vb, bg0, bg1, bg2, dimg, dalpha, T_final, n_contrib, gs, n_items);
    } else {
        __shared__ int s_next;
        for (;;) {
            __syncthreads();
            if (threadIdx.x == 0) s_next = atomicAdd(queue, 1);
            __syncthreads();
            const int q = s_next;
            if (q >= n_tiles) return;
            bwd_tile<NT, PPT>(order[q], ranges, pair_item, geo, col, conic_c, W, H, tw, TX, TY, vb, bg0, bg1, bg2, dimg, dalpha, T_final, n_contrib, gs, n_items);
        }
    }
}

int pixels_per_thread(const vbm_plan *p)
{
    const int npix = p->desc.tile_w * p->desc.tile_h;
    int ppt = p->desc.pixels_per_thread > 0 ? p->desc.pixels_per_thread : 2;
    while (ppt > 1 && npix / ppt < 32) ppt >>= 1;
    return ppt;
}

template <int NT, int PPT>
vbm_status launch_fwd(vbm_plan *p, int vb, int vc, const float bg[3], float *img, float *alpha, cudaStream_t st)
{
    const int n_tiles = vc * p->TX * p->TY;
    record_event(p->prof_ev[0], st);
    if (p->desc.flags & VBM_PLAN_PERSISTENT) {
        static int per_sm = 0;
        if (!per_sm) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_raster_fwd<NT, PPT, true>, NT, 0);
        const int grid = std::max(1, std::min(n_tiles, num_sms() * std::max(per_sm, 1)));
        k_raster_fwd<NT, PPT, true><<<grid, NT, 0, st>>>(
            p->tile_order, p->tile_queue, n_tiles, p->ranges, p->pair_item[p->pair_buf], p->geo, p->col, p->conic_c,
            p->desc.width, p->desc.height, p->desc.tile_w, p->TX, p->TY, vb, bg[0], bg[1], bg[2], img, alpha,
            p->T_final, p->n_contrib, p->prof_n_eval);
    } else {
        k_raster_fwd<NT, PPT, false><<<n_tiles, NT, 0, st>>>(
            nullptr, nullptr, n_tiles, p->ranges, p->pair_item[p->pair_buf], p->geo, p->col, p->conic_c,
            p->desc.width, p->desc.height, p->desc.tile_w, p->TX, p->TY, vb, bg[0], bg[1], bg[2], img, alpha,
            p->T_final, p->n_contrib, p->prof_n_eval);
    }
    VBM_LAUNCH("raster_fwd");
    record_event(p->prof_ev[1], st);
    note_launches(1);
    return VBM_OK;
}

template <int NT, int PPT>
vbm_status launch_bwd(vbm_plan *p, int vb, int vc, const float bg[3], const float *dimg, const float *dalpha,
                      cudaStream_t st)
{
    const int n_tiles = vc * p->TX * p->TY;
    record_event(p->prof_ev[2], st);
    if (p->desc.flags & VBM_PLAN_PERSISTENT) {
        static int per_sm = 0;
        if (!per_sm) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_raster_bwd<NT, PPT, true>, NT, 0);
        const int grid = std::max(1, std::min(n_tiles, num_sms() * std::max(per_sm, 1)));
        k_raster_bwd<NT, PPT, true><<<grid, NT, 0, st>>>(
            p->tile_order, p->tile_queue + 1, n_tiles, p->ranges, p->pair_item[p->pair_buf], p->geo, p->col,
            p->conic_c, p->desc.width, p->desc.height, p->desc.tile_w, p->TX, p->TY, vb, bg[0], bg[1], bg[2], dimg,
            dalpha, p->T_final, p->n_contrib, p->g_splat, p->last_items);
    } else {
        k_raster_bwd<NT, PPT, false><<<n_tiles, NT, 0, st>>>(
            nullptr, nullptr, n_tiles, p->ranges, p->pair_item[p->pair_buf], p->geo, p->col, p->conic_c,
            p->desc.width, p->desc.height, p->desc.tile_w, p->TX, p->TY, vb, bg[0], bg[1], bg[2], dimg, dalpha,
            p->T_final, p->n_contrib, p->g_splat, p->last_items);
    }
    VBM_LAUNCH("raster_bwd");
    record_event(p->prof_ev[3], st);
    note_launches(1);
    return VBM_OK;
}

// Dispatch on (pixels per tile, pixels per thread).
#define VBM_RASTER_DISPATCH(FN, ...)                                                          \
    switch (p->desc.tile_w * p->desc.tile_h * 8 + pixels_per_thread(p)) {                     \
        case 256 * 8 + 1: return FN<256, 1>(__VA_ARGS__);                                     \
        case 256 * 8 + 2: return FN<128, 2>(__VA_ARGS__);                                     \
        case 256 * 8 + 4: return FN<64, 4>(__VA_ARGS__);                                      \
        case 128 * 8 + 1: return FN<128, 1>(__VA_ARGS__);                                     \
        case 128 * 8 + 2: return FN<64, 2>(__VA_ARGS__);                                      \
        case 128 * 8 + 4: return FN<32, 4>(__VA_ARGS__);                                      \
        case 64 * 8 + 1: return FN<64, 1>(__VA_ARGS__);                                       \
        case 64 * 8 + 2: return FN<32, 2>(__VA_ARGS__);                                       \
        default: set_error("unsupported tile / pixels-per-thread combination"); return VBM_ERR_ARG; \
    }

}  // namespace

vbm_status raster_fwd(vbm_plan *p, int vb, int vc, const float bg[3], float *img, float *alpha, cudaStream_t st)
{
    VBM_RASTER_DISPATCH(launch_fwd, p, vb, vc, bg, img, alpha, st)
}

vbm_status raster_bwd(vbm_plan *p, const float *, int64_t, int vb, int vc, const float bg[3], const float *dimg,
                      const float *dalpha, float *, cudaStream_t st)
{
    VBM_CUDA(cudaMemsetAsync(p->g_splat, 0, sizeof(float) * 9 * p->last_items, st));
    VBM_RASTER_DISPATCH(launch_bwd, p, vb, vc, bg, dimg, dalpha, st)
}

}  // namespace vbm
