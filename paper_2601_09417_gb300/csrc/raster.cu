// Front-to-back alpha compositing of the binned splats and its reverse-order
// backward (Sec. 4.4, "as in" 3D Gaussian Splatting).
//
// One block per image tile (or a persistent grid pulling tiles from a work
// queue).  Each thread owns PPT consecutive pixels of one tile column.  The
// threads of a warp are split into lane groups of GL lanes (GL = 32, 16 or
// 8); a group owns a compact pixel block of the tile (8 x 4, 4 x 4 or 4 x 2
// thread positions for PPT = 1) and walks only the list entries whose
// alpha >= 1/255 ellipse can reach that block, so the groups of one warp work
// on different splats at the same time.  Two pixels' arithmetic is issued as
// packed FP32x2 operations (__ffma2_rn / __fmul2_rn / __fadd2_rn, sm_100+).
//
// A tile's depth-ordered list is staged through shared memory NT entries at a
// time.  While staging, each entry is tested against the tile: the minimum of
// its quadratic form over the rectangle of the tile's pixel centres gives the
// largest alpha any pixel of the tile can see; entries below the 1/255
// cut-off (with a 1e-3 margin in the exponent, far above rounding) are
// dropped and the rest compacted in list order.  The bounding box of each
// kept entry's alpha >= 1/255 ellipse is then intersected with the groups'
// pixel blocks, and every group compacts the entries that reach it into its
// own list of staged slots.  A dropped or unlisted entry would have been
// skipped by every pixel concerned, so the image, the saved state and the
// gradients are unchanged; the original list position travels with each
// entry for the contributor count.
//
// The conic is pre-scaled by -log2(e)/2 when staged, so the exponent is one
// ex2.approx.ftz per (pixel, splat) pair; its rounding sequence is fixed
// (explicit _rn operations) so the backward recomputes exactly the forward's
// alphas and skip decisions.  A pixel stops once its transmittance would
// fall below 1e-4; the block leaves the list when __syncthreads_count reports
// every pixel done.
//
// The backward walks each tile's list from the back, starting at the largest
// contributor count of the block (a group also drops entries beyond the
// largest contributor count of its own pixels), recovers the transmittance
// with a hardware reciprocal of (1 - alpha) and accumulates per-(view, splat)
// gradients: per splat, a group sums its nine partials over its lanes by a
// reduce-scatter (10 to 12 shuffles, skipped when no lane of the warp
// contributes), the lanes holding the sums add them to a shared-memory
// accumulator of the staged batch, and the batch is flushed to global memory
// with one atomic per nonzero value per (splat, tile).
#include "vbm_internal.h"

namespace vbm {
namespace {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;
constexpr float kHalfLog2e = -0.5f * kLog2e;   // scales A and C
constexpr float kNegLog2e = -kLog2e;           // scales B
constexpr float kCullMargin = 1e-3f;           // natural-log margin of the tile test
constexpr int kNV = 9;                         // gradient partials per (pixel, splat)

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Hardware reciprocal (one MUFU operation).  Used to undo a blend step,
// T_k = T_{k+1} / (1 - alpha_k) with 1 - alpha_k >= 0.01, so no operand is
// subnormal; its error is of the order of one FP32 rounding.
__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
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

// Thread rows per group by lane count (capped by the tile's thread rows).
__host__ __device__ constexpr int group_rows_default(int GL) { return GL == 8 ? 2 : 4; }

// Geometry of a tile and of this thread's lane group.  Threads form tw
// columns x (NT / tw) thread rows; a group covers GW columns x GR thread rows
// (GW * GR = GL), and groups are numbered row-major over the tile.
struct TileGeom {
    int vrel, px, py0;
    float pxc;
    float x0, x1, y0, y1;       // pixel-centre rectangle of the tile (clipped to the image)
    int tx0, ty0;               // tile origin in pixels
    int GW, GH, gpr;            // group block width and height in pixels, groups per block row
    int g, k;                   // this thread's group and lane in the group
};

template <int NT, int PPT, int GL>
__device__ __forceinline__ TileGeom tile_geom(int tile, int tw, int TX, int TY, int W, int H)
{
    constexpr int NPIX = NT * PPT;
    const int th = NPIX / tw;
    const int rows = NT / tw;
    const int GR = min(group_rows_default(GL), rows);
    TileGeom t;
    t.GW = GL / GR;
    t.GH = GR * PPT;
    t.gpr = tw / t.GW;
    const int tiles_per_view = TX * TY;
    t.vrel = tile / tiles_per_view;
    const int tt = tile - t.vrel * tiles_per_view;
    const int ty = tt / TX, tx = tt - ty * TX;
    t.tx0 = tx * tw;
    t.ty0 = ty * th;
    t.g = (int)threadIdx.x / GL;
    t.k = (int)threadIdx.x % GL;
    const int bx = t.g % t.gpr, by = t.g / t.gpr;
    t.px = t.tx0 + bx * t.GW + t.k % t.GW;
    t.py0 = t.ty0 + (by * GR + t.k / t.GW) * PPT;
    t.pxc = t.px + 0.5f;
    t.x0 = t.tx0 + 0.5f;
    t.x1 = min(t.tx0 + tw, W) - 0.5f;
    t.y0 = t.ty0 + 0.5f;
    t.y1 = min(t.ty0 + th, H) - 0.5f;
    return t;
}

// Groups whose pixel blocks the box [bx0, bx1] x [by0, by1] (pixel-centre
// coordinates) can reach: a bit mask over the NG groups of the tile.
template <int NG>
__device__ __forceinline__ uint32_t group_mask(const TileGeom &tg, float bx0, float bx1, float by0, float by1)
{
    const int n_rows = NG / tg.gpr;
    // block bx covers centres x0 + bx GW + [0, GW - 1]; likewise rows
    const float fx0 = (bx0 - tg.x0 - (float)(tg.GW - 1)) / (float)tg.GW;
    const float fx1 = (bx1 - tg.x0) / (float)tg.GW;
    const float fy0 = (by0 - tg.y0 - (float)(tg.GH - 1)) / (float)tg.GH;
    const float fy1 = (by1 - tg.y0) / (float)tg.GH;
    const int cx0 = max(0, (int)ceilf(fmaxf(fx0, -1.f)));
    const int cx1 = min(tg.gpr - 1, (int)floorf(fminf(fx1, (float)tg.gpr)));
    const int cy0 = max(0, (int)ceilf(fmaxf(fy0, -1.f)));
    const int cy1 = min(n_rows - 1, (int)floorf(fminf(fy1, (float)n_rows)));
    if (cx0 > cx1 || cy0 > cy1) return 0u;
    const uint64_t row = ((uint64_t(1) << (cx1 + 1)) - 1) & ~((uint64_t(1) << cx0) - 1);
    uint64_t m = 0;
    for (int r = cy0; r <= cy1; r++) m |= row << (r * tg.gpr);
    return (uint32_t)m;
}

// Shared-memory staging buffers of one batch of a tile list.
template <int NT, int GL>
struct Stage {
    static constexpr int NG = NT / GL;
    static constexpr int LSTRIDE = NT + 4;     // bytes per group list (spreads the groups over banks)
    float4 geo[NT];                            // u, v, A', B'
    float4 col[NT];                            // r, g, b, opacity
    float2 cp[NT];                             // C', list position (int bits)
    uint32_t mask[NT];                         // groups reached
    uint32_t item[NT];                         // item index (backward)
    uint8_t list[NG][LSTRIDE];                 // per group: staged slots reaching it, in list order
    int warp_cnt[NT / 32];
    int n;                                     // entries staged in this batch
};

// Stage entries [base, min(base + NT, end)) of a tile list: test each against
// the tile, compact the survivors in list order, and build every group's
// list.  gmax (backward) drops entries at or beyond a group's largest
// contributor count.  Returns this thread's group list length; all threads
// of the block must call it.
template <int NT, int GL>
__device__ __forceinline__ int stage_entries(int base, int end, int list_begin, const uint32_t *__restrict__ pair_item,
                                             const float4 *__restrict__ geo, const float4 *__restrict__ col,
                                             const float *__restrict__ conic_c, const TileGeom &tg,
                                             Stage<NT, GL> &s, const int *gmax)
{
    constexpr int NG = Stage<NT, GL>::NG;
    const int idx = base + (int)threadIdx.x;
    bool keep = false;
    float4 g = make_float4(0.f, 0.f, 0.f, 0.f), c = g;
    float cc = 0.f;
    uint32_t it = 0, msk = 0;
    if (idx < end) {
        it = pair_item[idx];
        g = geo[it];
        cc = conic_c[it];
        c = col[it];
        const float q = rect_min_quadratic(g.x, g.y, g.z, g.w, cc, tg.x0, tg.x1, tg.y0, tg.y1);
        const float tau = 2.f * (logf(255.f * c.w) + kCullMargin);
        keep = 0.5f * q <= 0.5f * tau;
        if (keep) {
            // bounding box of {q <= tau}: half-widths sqrt(tau C / det), sqrt(tau A / det) of the conic
            const float det = g.z * cc - g.w * g.w;
            const float hx = sqrtf(fmaxf(tau, 0.f) * cc / det) * 1.0001f + 1e-3f;
            const float hy = sqrtf(fmaxf(tau, 0.f) * g.z / det) * 1.0001f + 1e-3f;
            msk = group_mask<NG>(tg, g.x - hx, g.x + hx, g.y - hy, g.y + hy);
            if (gmax) {
                const int pos = idx - list_begin;
                for (uint32_t m = msk; m; m &= m - 1) {
                    const int gi = __ffs(m) - 1;
                    if (pos >= gmax[gi]) msk &= ~(1u << gi);
                }
            }
            keep = msk != 0;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t bal = __ballot_sync(0xffffffffu, keep);
    __syncthreads();            // the previous batch is no longer read
    if (lane == 0) s.warp_cnt[warp] = __popc(bal);
    __syncthreads();
    int before = 0, total = 0;
#pragma unroll
    for (int w = 0; w < NT / 32; w++) {
        const int cnt = s.warp_cnt[w];
        before += w < warp ? cnt : 0;
        total += cnt;
    }
    if (keep) {
        const int slot = before + __popc(bal & ((1u << lane) - 1u));
        s.geo[slot] = make_float4(g.x, g.y, g.z * kHalfLog2e, g.w * kNegLog2e);
        s.cp[slot] = make_float2(cc * kHalfLog2e, __int_as_float(idx - list_begin));
        s.col[slot] = c;
        s.mask[slot] = msk;
        s.item[slot] = it;
    }
    if (threadIdx.x == 0) s.n = total;
    __syncthreads();
    // each group scans the staged masks GL at a time and compacts its slots
    const int gshift = (GL == 32) ? 0 : (lane / GL) * GL;
    const uint32_t gbits = (GL == 32) ? 0xffffffffu : ((1u << GL) - 1u);
    const uint32_t below = (1u << tg.k) - 1u;
    int cnt = 0;
    for (int j0 = 0; j0 < total; j0 += GL) {        // uniform trip count
        const int j = j0 + tg.k;
        const bool in = j < total && ((s.mask[j] >> tg.g) & 1u);
        const uint32_t gb = (__ballot_sync(0xffffffffu, in) >> gshift) & gbits;
        if (in) s.list[tg.g][cnt + __popc(gb & below)] = (uint8_t)j;
        cnt += __popc(gb);
    }
    __syncthreads();
    return cnt;
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
template <int NT, int PPT, int GL, bool COLOR = true>
__device__ __forceinline__ void fwd_tile(const int tile, const int2 *__restrict__ ranges,
                                         const uint32_t *__restrict__ pair_item, const float4 *__restrict__ geo,
                                         const float4 *__restrict__ col, const float *__restrict__ conic_c, int W,
                                         int H, int tw, int TX, int TY, int vb, float bg0, float bg1, float bg2,
                                         float *__restrict__ img, float *__restrict__ alpha_out,
                                         float *__restrict__ T_final, int32_t *__restrict__ n_contrib,
                                         int32_t *__restrict__ n_eval, Stage<NT, GL> &s,
                                         PixState<PPT> *state = nullptr)
{
    static_assert(PPT == 1 || PPT % 2 == 0, "pixels per thread: 1 or even");
    constexpr int STEP = PPT == 1 ? 1 : 2;
    const TileGeom tg = tile_geom<NT, PPT, GL>(tile, tw, TX, TY, W, H);
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
        const int cnt = stage_entries<NT, GL>(base, rg.y, rg.x, pair_item, geo, col, conic_c, tg, s, nullptr);
        if (__all_sync(0xffffffffu, all_done)) continue;       // warp-uniform
        const int wmax = __reduce_max_sync(0xffffffffu, cnt);
        for (int i = 0; i < wmax; i++) {                       // no warp collectives inside
            if (i >= cnt) continue;
            const int j = s.list[tg.g][i];
            const float4 g = s.geo[j];
            const float2 cp = s.cp[j];
            const float4 c = s.col[j];
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

// One reduce-scatter step across lanes l and l ^ (1 << bit): of the N values
// of a lane, a lane with the bit clear keeps the lower half and one with the
// bit set keeps the upper half (zero-padded), each adding the partner's copy.
template <int N>
__device__ __forceinline__ void rs_half(const float (&in)[N], float (&out)[(N + 1) / 2], int bit)
{
    constexpr int HALF = (N + 1) / 2;
    const bool hi = (threadIdx.x >> bit) & 1;
#pragma unroll
    for (int i = 0; i < HALF; i++) {
        const float a = in[i], b = HALF + i < N ? in[HALF + i] : 0.f;
        const float send = hi ? a : b;
        const float keep = hi ? b : a;
        out[i] = keep + __shfl_xor_sync(0xffffffffu, send, 1 << bit);
    }
}

// Sum of nine values over a lane group, scattered over its lanes with
// halving steps (GL = 32: 12 shuffles, the last step a pair sum; GL = 16:
// 11 shuffles; GL = 8: 10 shuffles).  On return out[o] holds the group sum of
// value base + o for o < cnt, where (base, cnt) come from group_sum_layout.
template <int GL>
struct GroupSum {
    static constexpr int NOUT = GL == 8 ? 2 : 1;
    static constexpr int TOP = GL == 32 ? 4 : (GL == 16 ? 3 : 2);    // first lane bit halved
    static constexpr int STEPS = GL == 8 ? 3 : 4;
};

// Which values a lane holds after group_sum9: a lane whose bit is set keeps
// the upper ceil(N/2)-aligned half of its range (possibly all padding).
template <int GL>
__device__ __forceinline__ void group_sum_layout(int lane, int &base, int &cnt)
{
    int off = 0, c = kNV, n = kNV;
#pragma unroll
    for (int st = 0; st < GroupSum<GL>::STEPS; st++) {
        const int half = (n + 1) / 2;
        if ((lane >> (GroupSum<GL>::TOP - st)) & 1) {
            off += half;
            c = max(0, c - half);
        } else {
            c = min(c, half);
        }
        n = half;
    }
    base = off;
    cnt = (GL == 32 && (lane & 1)) ? 0 : c;    // odd lanes of the final pair sum repeat the even lane
}

template <int GL>
__device__ __forceinline__ void group_sum9(const float (&v)[kNV], float (&out)[GroupSum<GL>::NOUT])
{
    constexpr int T = GroupSum<GL>::TOP;
    float a5[5], a3[3], a2[2];
    rs_half<9>(v, a5, T);
    rs_half<5>(a5, a3, T - 1);
    rs_half<3>(a3, a2, T - 2);
    if constexpr (GL == 8) {
        out[0] = a2[0];
        out[1] = a2[1];
    } else {
        float a1[1];
        rs_half<2>(a2, a1, T - 3);
        if constexpr (GL == 32) out[0] = a1[0] + __shfl_xor_sync(0xffffffffu, a1[0], 1);
        else out[0] = a1[0];
    }
}

template <int NT, int PPT, int GL>
__device__ __forceinline__ void bwd_tile(const int tile, const int2 *__restrict__ ranges,
                                         const uint32_t *__restrict__ pair_item, const float4 *__restrict__ geo,
                                         const float4 *__restrict__ col, const float *__restrict__ conic_c, int W,
                                         int H, int tw, int TX, int TY, int vb, float bg0, float bg1, float bg2,
                                         const float *__restrict__ dimg, const float *__restrict__ dalpha,
                                         const float *__restrict__ T_final, const int32_t *__restrict__ n_contrib,
                                         float *__restrict__ gs, int64_t n_items, Stage<NT, GL> &s,
                                         float (&s_acc)[NT][kNV])
{
    constexpr int NG = Stage<NT, GL>::NG;
    __shared__ int s_gmax[NG];
    __shared__ int s_max;
    const TileGeom tg = tile_geom<NT, PPT, GL>(tile, tw, TX, TY, W, H);
    const int2 rg = ranges[tile];
    const int64_t HW = (int64_t)H * W;
    const int64_t v = vb + tg.vrel;
    float pyc[PPT], T[PPT], dC0[PPT], dC1[PPT], dC2[PPT], Q[PPT];
    int nc[PPT];
    int my_max = 0;
    PixState<PPT> rec;
    if (!T_final) {   // recompute mode: replay the forward decisions of this tile
        fwd_tile<NT, PPT, GL, false>(tile, ranges, pair_item, geo, col, conic_c, W, H, tw, TX, TY, vb, bg0, bg1, bg2,
                                     nullptr, nullptr, nullptr, nullptr, nullptr, s, &rec);
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
        // Q = sum over the splats behind (already walked) of (c . dL/dC) alpha T,
        // plus the background and alpha-output terms: dL/dalpha_k =
        // (c_k . dL/dC) T_k - Q / (1 - alpha_k)
        Q[k] = T[k] * (bg0 * dC0[k] + bg1 * dC1[k] + bg2 * dC2[k]) - dA * T[k];
        my_max = max(my_max, nc[k]);
    }
    // largest contributor count of each group and of the block
    int gm = my_max;
#pragma unroll
    for (int off = GL / 2; off > 0; off >>= 1) gm = max(gm, __shfl_xor_sync(0xffffffffu, gm, off));
    if (threadIdx.x == 0) s_max = 0;
    if (tg.k == 0) s_gmax[tg.g] = gm;
    __syncthreads();
    if (tg.k == 0) atomicMax(&s_max, gm);
    __syncthreads();
    const int max_nc = s_max;
    const int lane = threadIdx.x & 31;
    const int gshift = (GL == 32) ? 0 : (lane / GL) * GL;
    const uint32_t gbits = (GL == 32) ? 0xffffffffu : ((1u << GL) - 1u);
    int vbase, vcnt;
    group_sum_layout<GL>(lane, vbase, vcnt);
    for (int hi = max_nc; hi > 0; hi -= NT) {
        const int lo = max(0, hi - NT);
        const int cnt = stage_entries<NT, GL>(rg.x + lo, rg.x + hi, rg.x, pair_item, geo, col, conic_c, tg, s,
                                              s_gmax);
        const int wmax = __reduce_max_sync(0xffffffffu, cnt);
        for (int step = 0; step < wmax; step++) {   // back to front
            const int i = cnt - 1 - step;
            int j = 0;
            float acc[kNV];
#pragma unroll
            for (int q = 0; q < kNV; q++) acc[q] = 0.f;
            bool any = false;
            if (i >= 0) {
                j = s.list[tg.g][i];
                const float2 cp = s.cp[j];
                const int pos = __float_as_int(cp.y);
                const float4 g = s.geo[j];
                const float4 c = s.col[j];
                const float dx = __fsub_rn(g.x, tg.pxc);
                const float t0 = __fmul_rn(__fmul_rn(g.z, dx), dx);
                const float bdx = __fmul_rn(g.w, dx);
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
                        const float r_om = rcp_approx(1.f - alpha);
                        T[k] = T[k] * r_om;
                        const float wgt = alpha * T[k];
                        acc[6] += wgt * dC0[k];
                        acc[7] += wgt * dC1[k];
                        acc[8] += wgt * dC2[k];
                        const float cd = c.x * dC0[k] + c.y * dC1[k] + c.z * dC2[k];
                        const float dLda = cd * T[k] - Q[k] * r_om;
                        Q[k] += cd * wgt;
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
            }
            const uint32_t bal = __ballot_sync(0xffffffffu, any);
            if (!bal) continue;                          // warp-uniform
            float sum[GroupSum<GL>::NOUT];
            group_sum9<GL>(acc, sum);
            if ((bal >> gshift) & gbits) {
#pragma unroll
                for (int o = 0; o < GroupSum<GL>::NOUT; o++)
                    if (o < vcnt) atomicAdd(&s_acc[j][vbase + o], sum[o]);
            }
        }
        __syncthreads();
        // flush the batch: one global atomic per nonzero value, then clear
        for (int e = threadIdx.x; e < s.n * kNV; e += NT) {
            const int slot = e / kNV, q = e - slot * kNV;
            const float val = s_acc[slot][q];
            if (val != 0.f) {
                atomicAdd(&gs[(int64_t)q * n_items + s.item[slot]], val);
                s_acc[slot][q] = 0.f;
            }
        }
        __syncthreads();
    }
}

// Kernels: one block per tile, or (PERSIST) a grid of SMs x resident blocks
// whose blocks take tiles from an atomic queue in longest-list-first order.
template <int NT, int PPT, int GL, bool PERSIST>
__global__ void __launch_bounds__(NT)
    k_raster_fwd(const int *__restrict__ order, int *__restrict__ queue, int n_tiles, const int2 *__restrict__ ranges,
                 const uint32_t *__restrict__ pair_item, const float4 *__restrict__ geo,
                 const float4 *__restrict__ col, const float *__restrict__ conic_c, int W, int H, int tw, int TX,
                 int TY, int vb, float bg0, float bg1, float bg2, float *__restrict__ img,
                 float *__restrict__ alpha_out, float *__restrict__ T_final, int32_t *__restrict__ n_contrib,
                 int32_t *__restrict__ n_eval)
{
    __shared__ Stage<NT, GL> s;
    if constexpr (!PERSIST) {
        fwd_tile<NT, PPT, GL>(blockIdx.x, ranges, pair_item, geo, col, conic_c, W, H, tw, TX, TY, vb, bg0, bg1, bg2,
                              img, alpha_out, T_final, n_contrib, n_eval, s);
    } else {
        __shared__ int s_next;
        for (;;) {
            __syncthreads();
            if (threadIdx.x == 0) s_next = atomicAdd(queue, 1);
            __syncthreads();
            const int q = s_next;
            if (q >= n_tiles) return;
            fwd_tile<NT, PPT, GL>(order[q], ranges, pair_item, geo, col, conic_c, W, H, tw, TX, TY, vb, bg0, bg1,
                                  bg2, img, alpha_out, T_final, n_contrib, n_eval, s);
        }
    }
}

template <int NT, int PPT, int GL, bool PERSIST>
__global__ void __launch_bounds__(NT)
    k_raster_bwd(const int *__restrict__ order, int *__restrict__ queue, int n_tiles, const int2 *__restrict__ ranges,
                 const uint32_t *__restrict__ pair_item, const float4 *__restrict__ geo,
                 const float4 *__restrict__ col, const float *__restrict__ conic_c, int W, int H, int tw, int TX,
                 int TY, int vb, float bg0, float bg1, float bg2, const float *__restrict__ dimg,
                 const float *__restrict__ dalpha, const float *__restrict__ T_final,
                 const int32_t *__restrict__ n_contrib, float *__restrict__ gs, int64_t n_items)
{
    __shared__ Stage<NT, GL> s;
    __shared__ float s_acc[NT][kNV];
    for (int e = threadIdx.x; e < NT * kNV; e += NT) (&s_acc[0][0])[e] = 0.f;
    __syncthreads();
    if constexpr (!PERSIST) {
        bwd_tile<NT, PPT, GL>(blockIdx.x, ranges, pair_item, geo, col, conic_c, W, H, tw, TX, TY, vb, bg0, bg1, bg2,
                              dimg, dalpha, T_final, n_contrib, gs, n_items, s, s_acc);
    } else {
        __shared__ int s_next;
        for (;;) {
            __syncthreads();
            if (threadIdx.x == 0) s_next = atomicAdd(queue, 1);
            __syncthreads();
            const int q = s_next;
            if (q >= n_tiles) return;
            bwd_tile<NT, PPT, GL>(order[q], ranges, pair_item, geo, col, conic_c, W, H, tw, TX, TY, vb, bg0, bg1,
                                  bg2, dimg, dalpha, T_final, n_contrib, gs, n_items, s, s_acc);
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

int group_lanes(const vbm_plan *p) { return p->desc.group_lanes > 0 ? p->desc.group_lanes : 32; }

template <int NT, int PPT, int GL>
vbm_status launch_fwd(vbm_plan *p, int vb, int vc, const float bg[3], float *img, float *alpha, cudaStream_t st)
{
    const int n_tiles = vc * p->TX * p->TY;
    record_event(p->prof_ev[0], st);
    if (p->desc.flags & VBM_PLAN_PERSISTENT) {
        static int per_sm = 0;
        if (!per_sm) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_raster_fwd<NT, PPT, GL, true>, NT, 0);
        const int grid = std::max(1, std::min(n_tiles, num_sms() * std::max(per_sm, 1)));
        k_raster_fwd<NT, PPT, GL, true><<<grid, NT, 0, st>>>(
            p->tile_order, p->tile_queue, n_tiles, p->ranges, p->pair_item[p->pair_buf], p->geo, p->col, p->conic_c,
            p->desc.width, p->desc.height, p->desc.tile_w, p->TX, p->TY, vb, bg[0], bg[1], bg[2], img, alpha,
            p->T_final, p->n_contrib, p->prof_n_eval);
    } else {
        k_raster_fwd<NT, PPT, GL, false><<<n_tiles, NT, 0, st>>>(
            nullptr, nullptr, n_tiles, p->ranges, p->pair_item[p->pair_buf], p->geo, p->col, p->conic_c,
            p->desc.width, p->desc.height, p->desc.tile_w, p->TX, p->TY, vb, bg[0], bg[1], bg[2], img, alpha,
            p->T_final, p->n_contrib, p->prof_n_eval);
    }
    VBM_LAUNCH("raster_fwd");
    record_event(p->prof_ev[1], st);
    note_launches(1);
    return VBM_OK;
}

template <int NT, int PPT, int GL>
vbm_status launch_bwd(vbm_plan *p, int vb, int vc, const float bg[3], const float *dimg, const float *dalpha,
                      cudaStream_t st)
{
    const int n_tiles = vc * p->TX * p->TY;
    record_event(p->prof_ev[2], st);
    if (p->desc.flags & VBM_PLAN_PERSISTENT) {
        static int per_sm = 0;
        if (!per_sm) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_raster_bwd<NT, PPT, GL, true>, NT, 0);
        const int grid = std::max(1, std::min(n_tiles, num_sms() * std::max(per_sm, 1)));
        k_raster_bwd<NT, PPT, GL, true><<<grid, NT, 0, st>>>(
            p->tile_order, p->tile_queue + 1, n_tiles, p->ranges, p->pair_item[p->pair_buf], p->geo, p->col,
            p->conic_c, p->desc.width, p->desc.height, p->desc.tile_w, p->TX, p->TY, vb, bg[0], bg[1], bg[2], dimg,
            dalpha, p->T_final, p->n_contrib, p->g_splat, p->last_items);
    } else {
        k_raster_bwd<NT, PPT, GL, false><<<n_tiles, NT, 0, st>>>(
            nullptr, nullptr, n_tiles, p->ranges, p->pair_item[p->pair_buf], p->geo, p->col, p->conic_c,
            p->desc.width, p->desc.height, p->desc.tile_w, p->TX, p->TY, vb, bg[0], bg[1], bg[2], dimg, dalpha,
            p->T_final, p->n_contrib, p->g_splat, p->last_items);
    }
    VBM_LAUNCH("raster_bwd");
    record_event(p->prof_ev[3], st);
    note_launches(1);
    return VBM_OK;
}

// Dispatch on (pixels per tile, pixels per thread, lanes per group).
#define VBM_RASTER_CASES(FN, NPIX, GL, ...)                                                   \
    case (NPIX) * 64 + 1 * 8 + (GL) / 8: return FN<(NPIX), 1, (GL)>(__VA_ARGS__);             \
    case (NPIX) * 64 + 2 * 8 + (GL) / 8: return FN<(NPIX) / 2, 2, (GL)>(__VA_ARGS__);         \
    case (NPIX) * 64 + 4 * 8 + (GL) / 8: return FN<(NPIX) / 4, 4, (GL)>(__VA_ARGS__);

#define VBM_RASTER_DISPATCH(FN, ...)                                                                      \
    switch (p->desc.tile_w * p->desc.tile_h * 64 + pixels_per_thread(p) * 8 + group_lanes(p) / 8) {       \
        VBM_RASTER_CASES(FN, 256, 8, __VA_ARGS__)                                                         \
        VBM_RASTER_CASES(FN, 256, 16, __VA_ARGS__)                                                        \
        VBM_RASTER_CASES(FN, 256, 32, __VA_ARGS__)                                                        \
        VBM_RASTER_CASES(FN, 128, 8, __VA_ARGS__)                                                         \
        VBM_RASTER_CASES(FN, 128, 16, __VA_ARGS__)                                                        \
        VBM_RASTER_CASES(FN, 128, 32, __VA_ARGS__)                                                        \
        case 64 * 64 + 1 * 8 + 1: return FN<64, 1, 8>(__VA_ARGS__);                                       \
        case 64 * 64 + 2 * 8 + 1: return FN<32, 2, 8>(__VA_ARGS__);                                       \
        case 64 * 64 + 1 * 8 + 2: return FN<64, 1, 16>(__VA_ARGS__);                                      \
        case 64 * 64 + 2 * 8 + 2: return FN<32, 2, 16>(__VA_ARGS__);                                      \
        case 64 * 64 + 1 * 8 + 4: return FN<64, 1, 32>(__VA_ARGS__);                                      \
        case 64 * 64 + 2 * 8 + 4: return FN<32, 2, 32>(__VA_ARGS__);                                      \
        default: set_error("unsupported tile / pixels-per-thread / group-lanes combination"); return VBM_ERR_ARG; \
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
