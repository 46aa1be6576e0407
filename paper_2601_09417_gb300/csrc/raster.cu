// Front-to-back alpha compositing of the binned splats and its reverse-order
// backward (Sec. 4.4, "as in" 3D Gaussian Splatting).
//
// Work is split into warp regions: a warp owns 8 columns x 4 thread rows of a
// tile, each thread PPT consecutive pixels of its column, and walks the tile's
// depth-ordered list on its own (no block barriers), 32 entries per round:
// each lane loads one entry, tests it exactly against the warp region (the
// minimum of the splat's quadratic form over the rectangle of the region's
// pixel centres gives the largest alpha any of its pixels can see; entries
// below the 1/255 cut-off, with a 1e-3 margin in the exponent far above
// rounding, are dropped) and stores it in the warp's shared-memory slot.  The
// lanes of the warp form groups of GL lanes (GL = 32, 16, 8 or 4) that own
// 8 x 4, 4 x 4, 4 x 2 or 2 x 2 thread positions; a group keeps a 32-bit mask of the
// slots whose alpha >= 1/255 bounding box reaches its pixels and walks only
// those, so the groups of a warp composite different splats at the same
// time.  An entry a warp drops or a group skips would have been skipped by
// every pixel concerned, so images, saved state and gradients are unchanged;
// each staged entry carries its list position for the contributor count.
//
// The conic is pre-scaled by -log2(e)/2 when staged, so the exponent is one
// ex2.approx.ftz per (pixel, splat) pair; its rounding sequence is fixed
// (explicit _rn operations) so the backward recomputes exactly the forward's
// alphas and skip decisions.  A pixel stops once its transmittance would fall
// below 1e-4; a warp leaves the list when all its pixels have stopped.  Two
// pixels' arithmetic (PPT >= 2) is issued as packed FP32x2 operations
// (__ffma2_rn / __fmul2_rn / __fadd2_rn, sm_100+).
//
// The backward walks the list from the back, starting at the warp's largest
// contributor count (a group also drops entries beyond the largest count of
// its own pixels), recovers the transmittance with a hardware reciprocal of
// (1 - alpha) and accumulates per-(view, splat) gradients: per splat, a group
// sums its nine partials over its lanes by a reduce-scatter (8 to 12
// shuffles, skipped when no lane of the warp contributes), the lanes holding
// the sums add them to the warp's shared-memory accumulator for the round,
// and the round is flushed to the per-item gradient records with vector
// atomics (two float4 and one float per staged entry with a nonzero value),
// the partials' constant factors applied at the flush.
//
// Launch: blocks of kWarps warps; each warp takes work items (tile, region)
// either by its global warp index or, persistent, from an atomic queue whose
// items follow the tiles' longest-list-first order.  In persistent plans a
// tile whose list is longer than the segment length L is walked by the
// backward as independent units (tile, segment, region) of L entries, taken
// ahead of the whole tiles: the forward stores, per pixel still compositing
// at each segment boundary, the transmittance and the colour still to come
// (and, in recompute plans, the tile's final per-pixel state), from which a
// unit starts its walk; one warp's walk of a very long list otherwise
// outlasted the rest of the launch.  The backward may run its own pixels per
// thread and lane groups: its regions are independent of the forward's.
#include "vbm_internal.h"

namespace vbm {
namespace {

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;
constexpr float kHalfLog2e = -0.5f * kLog2e;   // scales A and C
constexpr float kNegLog2e = -kLog2e;           // scales B
constexpr int kNV = 9;                         // gradient partials per (pixel, splat)
constexpr int kWarps = 4;                      // warps per block
constexpr int kRegionCols = 8, kRegionRows = 4;   // thread positions of a warp region

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
// rectangle [x0, x1] x [y0, y1]: 0 inside, else the minimum over the (at most
// two) edges whose half-planes exclude the centre, each the clamped 1D
// minimiser (bc = B / C, ba = B / A precomputed); the binning's tile test
// (tile_min_q) gives the reason.
__device__ __forceinline__ float rect_min_quadratic(float u, float v, float A, float B, float C, float bc, float ba,
                                                    float x0, float x1, float y0, float y1)
{
    const bool left = u < x0, right = u > x1, below = v < y0, above = v > y1;
    if (!(left || right || below || above)) return 0.f;
    const float dx = (left ? x0 : x1) - u;
    const float dy = fminf(fmaxf(v - bc * dx, y0), y1) - v;
    const float qv = A * dx * dx + 2.f * B * dx * dy + C * dy * dy;
    const float ey = (below ? y0 : y1) - v;
    const float ex = fminf(fmaxf(u - ba * ey, x0), x1) - u;
    const float qh = A * ex * ex + 2.f * B * ex * ey + C * ey * ey;
    return fminf(left || right ? qv : 3.4e38f, below || above ? qh : 3.4e38f);
}

// Lane groups inside a warp region: GL lanes cover GW columns x GR thread rows.
template <int GL>
struct Groups {
    static_assert(GL == 4 || GL == 8 || GL == 16 || GL == 32, "lane groups of 4, 8, 16 or 32");
    static constexpr int GR = GL <= 8 ? 2 : 4;     // thread rows
    static constexpr int GW = GL / GR;              // columns: 4, 4, 8
    static constexpr int PER_ROW = kRegionCols / GW;
    static constexpr int NG = 32 / GL;              // groups per warp
};

// Geometry of a work item (tile, region) for this lane.
struct WarpGeom {
    int tile, vrel, px, py0;
    int pit0;                   // index of the lane's first pixel inside the tile (row-major, tile_w wide)
    float pxc;
    float x0, x1, y0, y1;       // pixel-centre rectangle of the region (clipped to the image)
    float gx0[8], gy0[8];       // first pixel centre of each group's block
    int g;                      // this lane's group
};

template <int PPT, int GL>
__device__ __forceinline__ WarpGeom warp_geom(int tile, int region, int tw, int th, int TX, int TY, int W, int H)
{
    using Gp = Groups<GL>;
    WarpGeom t;
    t.tile = tile;
    const int tiles_per_view = TX * TY;
    t.vrel = tile / tiles_per_view;
    const int tt = tile - t.vrel * tiles_per_view;
    const int ty = tt / TX, tx = tt - ty * TX;
    const int rpr = tw / kRegionCols;
    const int rx = region % rpr, ry = region / rpr;
    const int ox = tx * tw + rx * kRegionCols;
    const int oy = ty * th + ry * kRegionRows * PPT;
    const int lane = threadIdx.x & 31;
    t.g = lane / GL;
    const int k = lane % GL;
#pragma unroll
    for (int g = 0; g < Gp::NG; g++) {
        t.gx0[g] = ox + (g % Gp::PER_ROW) * Gp::GW + 0.5f;
        t.gy0[g] = oy + (g / Gp::PER_ROW) * Gp::GR * PPT + 0.5f;
    }
    t.px = ox + (t.g % Gp::PER_ROW) * Gp::GW + k % Gp::GW;
    t.py0 = oy + ((t.g / Gp::PER_ROW) * Gp::GR + k / Gp::GW) * PPT;
    t.pxc = t.px + 0.5f;
    t.pit0 = (t.py0 - ty * th) * tw + (t.px - tx * tw);
    t.x0 = ox + 0.5f;
    t.x1 = min(ox + kRegionCols, W) - 0.5f;
    t.y0 = oy + 0.5f;
    t.y1 = min(oy + kRegionRows * PPT, H) - 0.5f;
    return t;
}

// Shared-memory slots of one warp's round (entry j in slot j).
struct WarpSlots {
    float4 geo[32];         // u, v, A', B'
    float4 col[32];         // r, g, b, opacity
    float2 cp[32];          // C', list position + 1 (int bits)
    uint32_t item[32];
};

// Rounds of list entries the backward keeps in flight: their per-item data
// is copied asynchronously (cp.async) into shared memory while earlier
// rounds are processed, so the prefetch depth costs no registers.  Lane l
// copies, and later reads, entry l of a round.
constexpr int kStages = 3;

struct RawStages {
    float4 geo[kStages][32];
    float4 col[kStages][32];
    float4 cull[kStages][32];
    float cc[kStages][32];
    uint32_t it[kStages][32];
};

// One list entry's per-item data as loaded by a lane (it = kNoItem: none).
constexpr uint32_t kNoItem = 0xffffffffu;

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(a), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(a), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

// Wait until at most N of this thread's copy groups are still in flight.
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

struct Entry {
    uint32_t it;
    float4 g;       // u, v, A, B
    float4 c;       // r, g, b, opacity
    float4 cu;      // hx, hy, B / C, B / A
    float cc;       // C
};

__device__ __forceinline__ uint32_t load_index(const uint32_t *__restrict__ pair_item, int idx, int end)
{
    return idx < end ? pair_item[idx] : kNoItem;
}

__device__ __forceinline__ Entry gather_entry(uint32_t it, const SplatRec *__restrict__ rec)
{
    Entry e;
    e.it = it;
    if (it != kNoItem) {
        const SplatRec *r = rec + it;
        e.g = r->g;
        e.c = r->c;
        e.cu = r->cu;
        e.cc = r->x.x;
    } else {
        e.g = e.c = e.cu = make_float4(0.f, 0.f, 0.f, 0.f);
        e.cc = 0.f;
    }
    return e;
}

// Start copying the lane's entry `it` of a round into stage st; one copy
// group per round, empty when there is no entry.
__device__ __forceinline__ void stage_entry(RawStages &rs, int st, uint32_t it, const SplatRec *__restrict__ rec)
{
    const int lane = threadIdx.x & 31;
    rs.it[st][lane] = it;
    if (it != kNoItem) {
        const SplatRec *r = rec + it;
        cp_async16(&rs.geo[st][lane], &r->g);
        cp_async16(&rs.col[st][lane], &r->c);
        cp_async16(&rs.cull[st][lane], &r->cu);
        cp_async4(&rs.cc[st][lane], &r->x.x);
    }
    cp_async_commit();
}

// The lane's staged entry of stage st (its copies must have completed).
__device__ __forceinline__ Entry read_entry(const RawStages &rs, int st)
{
    const int lane = threadIdx.x & 31;
    Entry e;
    e.it = rs.it[st][lane];
    if (e.it != kNoItem) {
        e.g = rs.geo[st][lane];
        e.c = rs.col[st][lane];
        e.cu = rs.cull[st][lane];
        e.cc = rs.cc[st][lane];
    } else {
        e.g = e.c = e.cu = make_float4(0.f, 0.f, 0.f, 0.f);
        e.cc = 0.f;
    }
    return e;
}

// Test a lane's loaded entry (list position pos1 - 1) against the warp region
// and store it in the lane's slot.  Returns, for this lane's group, the mask
// of slots whose alpha >= 1/255 box reaches the group's pixels.  gmax
// (backward) holds each group's largest contributor count: entries beyond it
// are not listed for that group.
template <int PPT, int GL>
__device__ __forceinline__ uint32_t commit_entry(const Entry &e, int pos1, const WarpGeom &wg, WarpSlots &s,
                                                 const int *gmax)
{
    using Gp = Groups<GL>;
    const int lane = threadIdx.x & 31;
    uint32_t gbits = 0;       // bit g: entry reaches group g
    if (e.it != kNoItem) {
        const float4 g = e.g, cu = e.cu;
        const float q = rect_min_quadratic(g.x, g.y, g.z, g.w, e.cc, cu.z, cu.w, wg.x0, wg.x1, wg.y0, wg.y1);
        const float tau = 2.f * (__logf(255.f * e.c.w) + kCullMargin);
        if (0.5f * q <= 0.5f * tau) {
            const float bx0 = g.x - cu.x, bx1 = g.x + cu.x, by0 = g.y - cu.y, by1 = g.y + cu.y;
#pragma unroll
            for (int gi = 0; gi < Gp::NG; gi++) {
                const bool hit = bx1 >= wg.gx0[gi] && bx0 <= wg.gx0[gi] + (float)(Gp::GW - 1) &&
                                 by1 >= wg.gy0[gi] && by0 <= wg.gy0[gi] + (float)(Gp::GR * PPT - 1) &&
                                 (!gmax || pos1 <= gmax[gi]);
                gbits |= hit ? (1u << gi) : 0u;
            }
            if (gbits) {
                s.geo[lane] = make_float4(g.x, g.y, g.z * kHalfLog2e, g.w * kNegLog2e);
                s.cp[lane] = make_float2(e.cc * kHalfLog2e, __int_as_float(pos1));
                s.col[lane] = e.c;
                s.item[lane] = e.it;
            }
        }
    }
    uint32_t mine = 0;
#pragma unroll
    for (int gi = 0; gi < Gp::NG; gi++) {
        const uint32_t m = __ballot_sync(0xffffffffu, (gbits >> gi) & 1u);
        mine = gi == wg.g ? m : mine;
    }
    __syncwarp();
    return mine;
}

// Per-pixel compositing state of a thread's pixels after the forward walk.
template <int PPT>
struct PixState {
    float T[PPT];
    int last[PPT];
};

// Forward walk of one warp region.  COLOR = false computes only the per-pixel
// state (final transmittance and last contributor), with exactly the
// decisions of the full forward: the backward uses it when the state is not
// stored.
// The entries are prefetched in registers, or, with rs (the backward's replay),
// through its asynchronous shared-memory stages.
template <int PPT, int GL, bool COLOR = true, bool EVAL = false>
__device__ __forceinline__ void fwd_region(const WarpGeom &wg, const int2 *__restrict__ ranges,
                                           const uint32_t *__restrict__ pair_item, const SplatRec *__restrict__ rec, int W, int H, int vb, float bg0,
                                           float bg1, float bg2, float *__restrict__ img,
                                           float *__restrict__ alpha_out, float *__restrict__ T_final,
                                           int32_t *__restrict__ n_contrib, int32_t *__restrict__ n_eval,
                                           WarpSlots &s, PixState<PPT> *state = nullptr, RawStages *rs = nullptr,
                                           float4 *ck = nullptr, int seg_len = 0, int tw = 0, int tile_px = 0)
{
    static_assert(PPT == 1 || PPT % 2 == 0, "pixels per thread: 1 or even");
    constexpr int STEP = PPT == 1 ? 1 : 2;
    const int2 rg = ranges[wg.tile];
    float pyc[PPT], T[PPT], C0[PPT], C1[PPT], C2[PPT];
    int last[PPT], evaluated[PPT];
    bool inside[PPT], done[PPT];
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        const int py = wg.py0 + k;
        pyc[k] = py + 0.5f;
        inside[k] = wg.px < W && py < H;
        done[k] = !inside[k];
        T[k] = 1.f;
        C0[k] = C1[k] = C2[k] = 0.f;
        last[k] = 0;
        evaluated[k] = rg.y - rg.x;
    }
    // rounds of 32 entries, software-pipelined in registers: while round r is
    // composited, the lane's entries of rounds r + 1 and r + 2 and its index in
    // round r + 3 are in flight
    const int lane = threadIdx.x & 31;
    const int n_rounds = (rg.y - rg.x + 31) / 32;
    constexpr bool kAsync = !COLOR;
    Entry cur, nxt;
    uint32_t it_next;
    if constexpr (kAsync) {
#pragma unroll
        for (int d = 0; d < kStages - 1; d++)
            stage_entry(*rs, d, load_index(pair_item, rg.x + 32 * d + lane, rg.y), rec);
        it_next = load_index(pair_item, rg.x + 32 * (kStages - 1) + lane, rg.y);
    } else {
        cur = gather_entry(load_index(pair_item, rg.x + lane, rg.y), rec);
        nxt = gather_entry(load_index(pair_item, rg.x + 32 + lane, rg.y), rec);
        it_next = load_index(pair_item, rg.x + 64 + lane, rg.y);
    }
    for (int r = 0; r < n_rounds; r++) {
        bool all_done = true;
#pragma unroll
        for (int k = 0; k < PPT; k++) all_done &= done[k];
        if (__all_sync(0xffffffffu, all_done)) break;
        if (COLOR && ck && r > 0 && (32 * r) % seg_len == 0) {
            // segment boundary 32 r: state after the entries before it, for
            // the pixels still compositing (the others' backward starts from
            // their final state)
            float4 *slot = ck + (int64_t)((32 * r) / seg_len - 1) * tile_px;
#pragma unroll
            for (int k = 0; k < PPT; k++)
                if (!done[k]) slot[wg.pit0 + k * tw] = make_float4(T[k], C0[k], C1[k], C2[k]);
        }
        uint32_t m;
        if constexpr (kAsync) {
            stage_entry(*rs, (r + kStages - 1) % kStages, it_next, rec);
            it_next = load_index(pair_item, rg.x + 32 * (r + kStages) + lane, rg.y);
            cp_async_wait<kStages - 1>();
            m = commit_entry<PPT, GL>(read_entry(*rs, r % kStages), 32 * r + lane + 1, wg, s, nullptr);
        } else {
            const uint32_t it_after = load_index(pair_item, rg.x + 32 * (r + 3) + lane, rg.y);
            const Entry nxt2 = gather_entry(it_next, rec);
            m = commit_entry<PPT, GL>(cur, 32 * r + lane + 1, wg, s, nullptr);
            cur = nxt;
            nxt = nxt2;
            it_next = it_after;
        }
        while (m) {                                    // no warp collectives inside
            const int j = __ffs(m) - 1;
            m &= m - 1;
            const float4 g = s.geo[j];
            const float2 cp = s.cp[j];
            const float4 c = s.col[j];
            const int pos1 = __float_as_int(cp.y);
            const float dx = __fsub_rn(g.x, wg.pxc);
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
                    const float testT = __fmaf_rn(-alpha, T[kk], T[kk]);   // T (1 - alpha), one rounding
                    const bool term = cand && testT < kTMin;
                    const bool blend = cand && !term;
                    done[kk] = done[kk] || term;
                    if (EVAL && term) evaluated[kk] = pos1;
                    if (COLOR && blend) {
                        const float wgt = __fmul_rn(alpha, T[kk]);
                        C0[kk] = __fmaf_rn(c.x, wgt, C0[kk]);
                        C1[kk] = __fmaf_rn(c.y, wgt, C1[kk]);
                        C2[kk] = __fmaf_rn(c.z, wgt, C2[kk]);
                    }
                    T[kk] = blend ? testT : T[kk];
                    last[kk] = blend ? pos1 : last[kk];
                }
            }
        }
        __syncwarp();                                  // slots are rewritten next round
    }
    if constexpr (kAsync) cp_async_wait<0>();          // no copy in flight into the next user's stages
    if (state) {
#pragma unroll
        for (int k = 0; k < PPT; k++) {
            state->T[k] = T[k];
            state->last[k] = last[k];
        }
    }
    if (!COLOR) return;
    const int64_t HW = (int64_t)H * W;
    const int64_t v = vb + wg.vrel;
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        if (!inside[k]) continue;
        if (ck) {
            // checkpoints written for this pixel (boundaries before its last
            // contributor): colour so far -> colour still to come
            for (int b = seg_len; b < last[k]; b += seg_len) {
                float4 *a = ck + (int64_t)(b / seg_len - 1) * tile_px + wg.pit0 + k * tw;
                const float4 c = *a;
                *a = make_float4(c.x, C0[k] - c.y, C1[k] - c.z, C2[k] - c.w);
            }
            if (!T_final) {   // no per-pixel state kept: the tile's final state after its boundaries
                const int nseg = (rg.y - rg.x + seg_len - 1) / seg_len;
                ck[(int64_t)(nseg - 1) * tile_px + wg.pit0 + k * tw] =
                    make_float4(T[k], __int_as_float(last[k]), 0.f, 0.f);
            }
        }
        const int64_t pix = (int64_t)(wg.py0 + k) * W + wg.px;
        img[(v * 3 + 0) * HW + pix] = C0[k] + T[k] * bg0;
        img[(v * 3 + 1) * HW + pix] = C1[k] + T[k] * bg1;
        img[(v * 3 + 2) * HW + pix] = C2[k] + T[k] * bg2;
        if (alpha_out) alpha_out[v * HW + pix] = 1.f - T[k];
        if (T_final) T_final[v * HW + pix] = T[k];
        if (n_contrib) n_contrib[v * HW + pix] = last[k];
        if (EVAL) n_eval[v * HW + pix] = evaluated[k];
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
// 11 shuffles; GL = 8: 10 shuffles; GL = 4: 8 shuffles).  On return out[o]
// holds the group sum of value base + o for o < cnt, where (base, cnt) come
// from group_sum_layout.
template <int GL>
struct GroupSum {
    static constexpr int NOUT = GL == 4 ? 3 : (GL == 8 ? 2 : 1);
    static constexpr int TOP = GL == 32 ? 4 : (GL == 16 ? 3 : (GL == 8 ? 2 : 1));   // first lane bit halved
    static constexpr int STEPS = GL == 4 ? 2 : (GL == 8 ? 3 : 4);
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
    if constexpr (GL == 4) {
        out[0] = a3[0];
        out[1] = a3[1];
        out[2] = a3[2];
        return;
    }
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

// One backward step of a lane for splat slot j over its PPT pixels (PPT
// even), as pairs of pixels in packed FP32x2 operations and without
// branches: a pixel that does not blend this splat (beyond its last
// contributor, power > 0 or alpha < 1/255) gets zero weight and keeps its
// T and Q.  The exponent and alpha are the forward's, operation for
// operation (dy = g.y + (-pyc) equals g.y - pyc exactly), so the decisions
// are the forward's.  Writes the nine partials of this lane's pixels to acc
// (du, dv, dA, dB, dC, dopacity, dr, dg, db; conic terms in the natural-log
// parameterisation), du and dv without their factor ln 2 and dA and dC
// without their factor -1/2 (the round's flush applies them once per splat),
// and returns whether any pixel blended.
template <int PPT>
__device__ __forceinline__ bool pair_step(const WarpSlots &s, int j, float pxc, const float2 (&npyc)[PPT / 2],
                                          const int (&nc)[PPT], float (&T)[PPT], float (&Q)[PPT],
                                          const float (&dC0)[PPT], const float (&dC1)[PPT],
                                          const float (&dC2)[PPT], float (&acc)[kNV])
{
    const float2 cp = s.cp[j];
    const int pos1 = __float_as_int(cp.y);
    const float4 g = s.geo[j];
    const float4 c = s.col[j];
    const float dx = __fsub_rn(g.x, pxc);
    const float t0 = __fmul_rn(__fmul_rn(g.z, dx), dx);
    const float bdx = __fmul_rn(g.w, dx);
    const float2 a_dy = make_float2(g.w, g.w);                  // du: 2 A' dx + B' dy
    const float2 a_c = make_float2(2.f * g.z * dx, 2.f * g.z * dx);
    const float2 b_dy = make_float2(2.f * cp.x, 2.f * cp.x);    // dv: 2 C' dy + B' dx
    const float2 b_c = make_float2(g.w * dx, g.w * dx);
    bool any = false;
    float2 s_u = make_float2(0.f, 0.f), s_v = s_u, s_pw = s_u, s_dy = s_u, s_dy2 = s_u, s_G = s_u;
    float2 s_r = s_u, s_g = s_u, s_b = s_u;
#pragma unroll
    for (int h = 0; h < PPT / 2; h++) {
        const int k = 2 * h;
        const float2 dy = __fadd2_rn(make_float2(g.y, g.y), npyc[h]);
        const float2 t = __ffma2_rn(__fmul2_rn(make_float2(cp.x, cp.x), dy), dy, make_float2(t0, t0));
        const float2 p2 = __ffma2_rn(make_float2(bdx, bdx), dy, t);
        const float2 G = make_float2(ex2_approx(p2.x), ex2_approx(p2.y));
        const float2 raw = __fmul2_rn(make_float2(c.w, c.w), G);
        const float al0 = fminf(kAlphaMax, raw.x), al1 = fminf(kAlphaMax, raw.y);
        const bool v0 = pos1 <= nc[k] && p2.x <= 0.f && al0 >= kAlphaMin;
        const bool v1 = pos1 <= nc[k + 1] && p2.y <= 0.f && al1 >= kAlphaMin;
        any |= v0 | v1;
        const float2 alpha = make_float2(v0 ? al0 : 0.f, v1 ? al1 : 0.f);
        // r_om = 1 / (1 - alpha) for a blended pixel, 1 otherwise (T unchanged)
        const float2 r_om = make_float2(v0 ? rcp_approx(1.f - al0) : 1.f, v1 ? rcp_approx(1.f - al1) : 1.f);
        float2 Tk = __fmul2_rn(make_float2(T[k], T[k + 1]), r_om);
        const float2 wgt = __fmul2_rn(alpha, Tk);
        const float2 d0 = make_float2(dC0[k], dC0[k + 1]), d1 = make_float2(dC1[k], dC1[k + 1]);
        const float2 d2 = make_float2(dC2[k], dC2[k + 1]);
        s_r = h == 0 ? __fmul2_rn(wgt, d0) : __ffma2_rn(wgt, d0, s_r);
        s_g = h == 0 ? __fmul2_rn(wgt, d1) : __ffma2_rn(wgt, d1, s_g);
        s_b = h == 0 ? __fmul2_rn(wgt, d2) : __ffma2_rn(wgt, d2, s_b);
        const float2 cd = __ffma2_rn(make_float2(c.z, c.z), d2,
                                     __ffma2_rn(make_float2(c.y, c.y), d1, __fmul2_rn(make_float2(c.x, c.x), d0)));
        float2 Qk = make_float2(Q[k], Q[k + 1]);
        const float2 dLda = __ffma2_rn(cd, Tk, __fmul2_rn(Qk, make_float2(-r_om.x, -r_om.y)));
        Qk = __ffma2_rn(cd, wgt, Qk);
        // the 0.99 clamp passes no gradient to the opacity and the exponent
        const bool g0 = v0 && raw.x < kAlphaMax, g1 = v1 && raw.y < kAlphaMax;
        const float2 dLdaG = __fmul2_rn(dLda, G), dpw = __fmul2_rn(dLda, raw);
        const float2 dG = make_float2(g0 ? dLdaG.x : 0.f, g1 ? dLdaG.y : 0.f);
        const float2 dpow = make_float2(g0 ? dpw.x : 0.f, g1 ? dpw.y : 0.f);
        if (h == 0) {      // the first pair starts the sums
            s_G = dG;
            s_u = __fmul2_rn(dpow, __ffma2_rn(a_dy, dy, a_c));
            s_v = __fmul2_rn(dpow, __ffma2_rn(b_dy, dy, b_c));
            s_pw = dpow;
            s_dy = __fmul2_rn(dpow, dy);
            s_dy2 = __fmul2_rn(dpow, __fmul2_rn(dy, dy));
        } else {
            s_G = __fadd2_rn(s_G, dG);
            s_u = __ffma2_rn(dpow, __ffma2_rn(a_dy, dy, a_c), s_u);
            s_v = __ffma2_rn(dpow, __ffma2_rn(b_dy, dy, b_c), s_v);
            s_pw = __fadd2_rn(s_pw, dpow);
            s_dy = __ffma2_rn(dpow, dy, s_dy);
            s_dy2 = __ffma2_rn(dpow, __fmul2_rn(dy, dy), s_dy2);
        }
        T[k] = Tk.x;
        T[k + 1] = Tk.y;
        Q[k] = Qk.x;
        Q[k + 1] = Qk.y;
    }
    acc[0] = s_u.x + s_u.y;
    acc[1] = s_v.x + s_v.y;
    acc[2] = dx * dx * (s_pw.x + s_pw.y);
    acc[3] = -dx * (s_dy.x + s_dy.y);
    acc[4] = s_dy2.x + s_dy2.y;
    acc[5] = s_G.x + s_G.y;
    acc[6] = s_r.x + s_r.y;
    acc[7] = s_g.x + s_g.y;
    acc[8] = s_b.x + s_b.y;
    return any;
}

template <int PPT, int GL>
__device__ __forceinline__ void bwd_region(const WarpGeom &wg, const int2 *__restrict__ ranges,
                                           const uint32_t *__restrict__ pair_item, const SplatRec *__restrict__ rec, int W, int H, int vb, float bg0,
                                           float bg1, float bg2, const float *__restrict__ dimg,
                                           const float *__restrict__ dalpha, const float *__restrict__ T_final,
                                           const int32_t *__restrict__ n_contrib, float *__restrict__ gs,
                                           WarpSlots &s, RawStages &rs, float (&acc_s)[32][kNV], int seg = -1,
                                           const float4 *__restrict__ ck = nullptr, int seg_len = 0, int tw = 0,
                                           int tile_px = 0)
{
    using Gp = Groups<GL>;
    const int2 rg = ranges[wg.tile];
    // list positions [pa, pb) of this work unit: a segment, or the whole list
    const int len = rg.y - rg.x;
    const int pa = seg >= 0 ? seg * seg_len : 0;
    const int pb = seg >= 0 ? min(pa + seg_len, len) : len;
    const float4 *ck_end = seg >= 0 && pb < len ? ck + (int64_t)seg * tile_px : nullptr;   // boundary pb
    const int64_t HW = (int64_t)H * W;
    const int64_t v = vb + wg.vrel;
    const int lane = threadIdx.x & 31;
    float pyc[PPT], T[PPT], dC0[PPT], dC1[PPT], dC2[PPT], Q[PPT];
    int nc[PPT];
    int my_max = 0;
    PixState<PPT> replay;
    if (!T_final && seg < 0)   // recompute mode, whole list: replay the forward decisions of this region
        fwd_region<PPT, GL, false>(wg, ranges, pair_item, rec, W, H, vb, bg0, bg1, bg2, nullptr,
                                   nullptr, nullptr, nullptr, nullptr, s, &replay, &rs);
#pragma unroll
    for (int k = 0; k < PPT; k++) {
        const int py = wg.py0 + k;
        pyc[k] = py + 0.5f;
        T[k] = 1.f;
        dC0[k] = dC1[k] = dC2[k] = 0.f;
        nc[k] = 0;
        float dA = 0.f;
        if (wg.px < W && py < H) {
            const int64_t pix = (int64_t)py * W + wg.px;
            if (T_final) {
                T[k] = T_final[v * HW + pix];
                nc[k] = n_contrib[v * HW + pix];
            } else if (seg >= 0) {   // recompute mode, segmented tile: the state the forward kept for it
                const float4 f = ck[(int64_t)((len + seg_len - 1) / seg_len - 1) * tile_px + wg.pit0 + k * tw];
                T[k] = f.x;
                nc[k] = __float_as_int(f.y);
            } else {
                T[k] = replay.T[k];
                nc[k] = replay.last[k];
            }
            dC0[k] = dimg[(v * 3 + 0) * HW + pix];
            dC1[k] = dimg[(v * 3 + 1) * HW + pix];
            dC2[k] = dimg[(v * 3 + 2) * HW + pix];
            if (dalpha) dA = dalpha[v * HW + pix];
        }
        // Q = sum over the splats behind (already walked) of (c . dL/dC) alpha T,
        // plus the background and alpha-output terms: dL/dalpha_k =
        // (c_k . dL/dC) T_k - Q / (1 - alpha_k)
        Q[k] = T[k] * (bg0 * dC0[k] + bg1 * dC1[k] + bg2 * dC2[k]) - dA * T[k];
        if (ck_end && pb < nc[k]) {
            // the pixel still composited at pb: start from the transmittance
            // there, with the colour still to come in Q
            const float4 c = ck_end[wg.pit0 + k * tw];
            T[k] = c.x;
            Q[k] += c.y * dC0[k] + c.z * dC1[k] + c.w * dC2[k];
        }
        my_max = max(my_max, nc[k]);
    }
    // -(pixel centre y) of each pixel pair, for the packed step
    float2 npyc[(PPT + 1) / 2];
#pragma unroll
    for (int k = 0; k + 1 < PPT; k += 2) npyc[k / 2] = make_float2(-pyc[k], -pyc[k + 1]);
    // largest contributor count of each group and of the warp
    int gm = my_max;
#pragma unroll
    for (int off = GL / 2; off > 0; off >>= 1) gm = max(gm, __shfl_xor_sync(0xffffffffu, gm, off));
    int gmax[Gp::NG];
#pragma unroll
    for (int gi = 0; gi < Gp::NG; gi++) gmax[gi] = __shfl_sync(0xffffffffu, gm, gi * GL);
    const int wtop = min(pb, __reduce_max_sync(0xffffffffu, gm));   // walk positions [pa, wtop)
    int vbase, vcnt;
    group_sum_layout<GL>(lane, vbase, vcnt);
    const uint32_t gmask = GL == 32 ? 0xffffffffu : (((1u << GL) - 1u) << (wg.g * GL));
    // rounds from the back: round r holds list positions [max(pa, wtop - 32 (r + 1)), wtop - 32 r),
    // software-pipelined as in the forward
    const int n_rounds = wtop > pa ? (wtop - pa + 31) / 32 : 0;
    auto round_lo = [&](int r) { return max(pa, wtop - 32 * (r + 1)); };
    auto round_idx = [&](int r) { return rg.x + round_lo(r) + lane; };
    auto round_end = [&](int r) { return rg.x + wtop - 32 * r; };
    auto round_item = [&](int r) { return r < n_rounds ? load_index(pair_item, round_idx(r), round_end(r)) : kNoItem; };
#pragma unroll
    for (int d = 0; d < kStages - 1; d++) stage_entry(rs, d, round_item(d), rec);
    uint32_t it_next = round_item(kStages - 1);
    for (int r = 0; r < n_rounds; r++) {
        stage_entry(rs, (r + kStages - 1) % kStages, it_next, rec);
        it_next = round_item(r + kStages);
        cp_async_wait<kStages - 1>();
        const Entry cur = read_entry(rs, r % kStages);
        uint32_t m = commit_entry<PPT, GL>(cur, round_lo(r) + lane + 1, wg, s, gmax);
        const int steps = __reduce_max_sync(0xffffffffu, __popc(m));
        for (int step = 0; step < steps; step++) {   // back to front
            int j = 0;
            float acc[kNV];
#pragma unroll
            for (int q = 0; q < kNV; q++) acc[q] = 0.f;
            bool any = false;
            if constexpr (PPT % 2 == 0) {
                if (m) {
                    j = 31 - __clz(m);
                    m &= ~(1u << j);
                    any = pair_step<PPT>(s, j, wg.pxc, npyc, nc, T, Q, dC0, dC1, dC2, acc);
                }
            } else if (m) {
                j = 31 - __clz(m);
                m &= ~(1u << j);
                const float2 cp = s.cp[j];
                const int pos1 = __float_as_int(cp.y);
                const float4 g = s.geo[j];
                const float4 c = s.col[j];
                const float dx = __fsub_rn(g.x, wg.pxc);
                const float t0 = __fmul_rn(__fmul_rn(g.z, dx), dx);
                const float bdx = __fmul_rn(g.w, dx);
#pragma unroll
                for (int k = 0; k < PPT; k++) {
                    if (pos1 > nc[k]) continue;
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
                            acc[0] += dpow * (2.f * g.z * dx + g.w * dy);
                            acc[1] += dpow * (2.f * cp.x * dy + g.w * dx);
                            acc[2] += dpow * (dx * dx);
                            acc[3] += dpow * (-dx * dy);
                            acc[4] += dpow * (dy * dy);
                        }
                    }
                }
            }
            const uint32_t bal = __ballot_sync(0xffffffffu, any);
            if (!bal) continue;                          // warp-uniform
            float sum[GroupSum<GL>::NOUT];
            group_sum9<GL>(acc, sum);
            if (bal & gmask) {
#pragma unroll
                for (int o = 0; o < GroupSum<GL>::NOUT; o++)
                    if (o < vcnt) atomicAdd(&acc_s[j][vbase + o], sum[o]);
            }
        }
        __syncwarp();
        // flush the round: the lane of slot l adds its entry's sums to the item's record
        float a[kNV];
        bool nz = false;
#pragma unroll
        for (int q = 0; q < kNV; q++) {
            a[q] = acc_s[lane][q];
            nz |= a[q] != 0.f;
            acc_s[lane][q] = 0.f;
        }
        if (nz) {
            // the constant factors the step leaves out: ln 2 of the base-2
            // exponent in du and dv, -1/2 in dA and dC
            a[0] *= kLn2;
            a[1] *= kLn2;
            a[2] *= -0.5f;
            a[4] *= -0.5f;
            float *rec_g = gs + (int64_t)s.item[lane] * kGradStride;
            atomicAdd(reinterpret_cast<float4 *>(rec_g), make_float4(a[0], a[1], a[2], a[3]));
            atomicAdd(reinterpret_cast<float4 *>(rec_g + 4), make_float4(a[4], a[5], a[6], a[7]));
            atomicAdd(rec_g + 8, a[8]);
        }
        __syncwarp();
    }
    cp_async_wait<0>();
}

// Work item of a warp: the global warp index once, or items from the queue
// (PERSIST).  Returns false when there is no item left.
template <bool PERSIST>
__device__ __forceinline__ bool next_item(int &q, int w_global, int n_items_w, int *queue, bool first)
{
    if constexpr (!PERSIST) {
        q = first ? w_global : n_items_w;
    } else {
        int t = 0;
        if ((threadIdx.x & 31) == 0) t = atomicAdd(queue, 1);
        q = __shfl_sync(0xffffffffu, t, 0);
    }
    return q < n_items_w;
}

template <int PPT, int GL, bool PERSIST, bool EVAL>
__global__ void __launch_bounds__(kWarps * 32)
    k_raster_fwd(const int *__restrict__ order, int *__restrict__ queue, int n_items_w, int n_regions,
                 const int2 *__restrict__ ranges, const uint32_t *__restrict__ pair_item,
                 const SplatRec *__restrict__ rec, int W, int H, int tw, int th, int TX, int TY, int vb, float bg0,
                 float bg1, float bg2, float *__restrict__ img, float *__restrict__ alpha_out,
                 float *__restrict__ T_final, int32_t *__restrict__ n_contrib, int32_t *__restrict__ n_eval,
                 float4 *__restrict__ ckpt, const int *__restrict__ ckpt_base, int seg_len)
{
    __shared__ WarpSlots slots[kWarps];
    WarpSlots &s = slots[threadIdx.x >> 5];
    const int w_global = blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int tile_px = tw * th;
    int q;
    for (bool first = true; next_item<PERSIST>(q, w_global, n_items_w, queue, first); first = false) {
        const int tile = PERSIST ? order[q / n_regions] : q / n_regions;
        const WarpGeom wg = warp_geom<PPT, GL>(tile, q % n_regions, tw, th, TX, TY, W, H);
        if (wg.x0 > wg.x1 || wg.y0 > wg.y1) continue;            // region outside the image
        const int cb = ckpt_base ? ckpt_base[tile] : -1;
        fwd_region<PPT, GL, true, EVAL>(wg, ranges, pair_item, rec, W, H, vb, bg0, bg1, bg2, img, alpha_out,
                            T_final, n_contrib, n_eval, s, nullptr, nullptr,
                            cb >= 0 ? ckpt + (int64_t)cb * tile_px : nullptr, seg_len, tw, tile_px);
    }
}

template <int PPT, int GL, bool PERSIST>
__global__ void __launch_bounds__(kWarps * 32)
    k_raster_bwd(const int *__restrict__ order, int *__restrict__ queue, int n_items_w, int n_regions,
                 const int2 *__restrict__ ranges, const uint32_t *__restrict__ pair_item,
                 const SplatRec *__restrict__ rec, int W, int H, int tw, int th, int TX, int TY, int vb, float bg0,
                 float bg1, float bg2, const float *__restrict__ dimg, const float *__restrict__ dalpha,
                 const float *__restrict__ T_final, const int32_t *__restrict__ n_contrib, float *__restrict__ gs,
                 const int *__restrict__ seg_count, const int2 *__restrict__ seg_units,
                 const float4 *__restrict__ ckpt, const int *__restrict__ ckpt_base, int seg_len)
{
    __shared__ WarpSlots slots[kWarps];
    __shared__ RawStages raw[kWarps];
    __shared__ float acc_s[kWarps][32][kNV];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSlots &s = slots[w];
#pragma unroll
    for (int q = 0; q < kNV; q++) acc_s[w][lane][q] = 0.f;
    __syncwarp();
    const int w_global = blockIdx.x * kWarps + w;
    const int tile_px = tw * th;
    // work units: the segments of the segmented tiles (placed first in the
    // order), then every other tile whole in the order's sequence
    int n_units = 0, n_seg_tiles = 0;
    if (seg_units) {
        n_units = seg_count[kQSegUnits];
        n_seg_tiles = seg_count[kQSegTiles];
        n_items_w += (n_units - n_seg_tiles) * n_regions;
    }
    int q;
    for (bool first = true; next_item<PERSIST>(q, w_global, n_items_w, queue, first); first = false) {
        const int u = q / n_regions;
        int tile, seg = -1;
        if (u < n_units) {
            const int2 su = seg_units[u];
            tile = su.x;
            seg = su.y;
        } else {
            tile = PERSIST ? order[u - n_units + n_seg_tiles] : u;
        }
        const WarpGeom wg = warp_geom<PPT, GL>(tile, q - u * n_regions, tw, th, TX, TY, W, H);
        if (wg.x0 > wg.x1 || wg.y0 > wg.y1) continue;
        bwd_region<PPT, GL>(wg, ranges, pair_item, rec, W, H, vb, bg0, bg1, bg2, dimg, dalpha,
                            T_final, n_contrib, gs, s, raw[w], acc_s[w], seg,
                            seg >= 0 ? ckpt + (int64_t)ckpt_base[tile] * tile_px : nullptr, seg_len, tw, tile_px);
    }
}

// Pixels per thread and lanes per group of the forward (bwd = false) or the
// backward compositing kernel; the backward takes the forward's unless the
// plan sets its own.  Each kernel's warp regions are its own: the backward
// reads only per-pixel state and tile-indexed checkpoints of the forward.
int pixels_per_thread(const vbm_plan *p, bool bwd = false)
{
    const int th = p->desc.tile_h;
    const int want = bwd && p->desc.bwd_pixels_per_thread > 0 ? p->desc.bwd_pixels_per_thread
                                                               : p->desc.pixels_per_thread;
    int ppt = want > 0 ? want : 2;
    while (ppt > 1 && th % (kRegionRows * ppt) != 0) ppt >>= 1;
    return ppt;
}

int group_lanes(const vbm_plan *p, bool bwd = false)
{
    const int want = bwd && p->desc.bwd_group_lanes > 0 ? p->desc.bwd_group_lanes : p->desc.group_lanes;
    return want > 0 ? want : 32;
}

int regions_per_tile(const vbm_plan *p, int ppt)
{
    return (p->desc.tile_w / kRegionCols) * (p->desc.tile_h / (kRegionRows * ppt));
}

template <typename K>
int persistent_grid(K kernel, int n_items_w)
{
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kWarps * 32, 0);
    const int blocks_needed = (n_items_w + kWarps - 1) / kWarps;
    return std::max(1, std::min(blocks_needed, num_sms() * std::max(per_sm, 1)));
}

template <int PPT, int GL>
vbm_status launch_fwd(vbm_plan *p, int vb, int vc, const float bg[3], float *img, float *alpha, cudaStream_t st)
{
    const int n_tiles = vc * p->TX * p->TY;
    const int nr = regions_per_tile(p, PPT);
    const int n_items_w = n_tiles * nr;
    record_event(p->prof_ev[0], st);
    // the evaluated-entry count (a profiling output) is compiled only into the
    // variants launched while that hook is set
    const bool eval = p->prof_n_eval != nullptr;
    int32_t *nc_out = p->n_contrib ? p->n_contrib : p->prof_n_contrib;
    if (p->desc.flags & VBM_PLAN_PERSISTENT) {
        auto kernel = eval ? k_raster_fwd<PPT, GL, true, true> : k_raster_fwd<PPT, GL, true, false>;
        const int grid = persistent_grid(kernel, n_items_w);
        kernel<<<grid, kWarps * 32, 0, st>>>(p->tile_order, p->tile_queue, n_items_w, nr, p->ranges, p->pair_item,
                                             p->rec, p->desc.width, p->desc.height, p->desc.tile_w, p->desc.tile_h,
                                             p->TX, p->TY, vb, bg[0], bg[1], bg[2], img, alpha, p->T_final, nc_out,
                                             p->prof_n_eval, p->ckpt, p->seg_len ? p->ckpt_base : nullptr,
                                             p->seg_len);
    } else {
        auto kernel = eval ? k_raster_fwd<PPT, GL, false, true> : k_raster_fwd<PPT, GL, false, false>;
        kernel<<<(n_items_w + kWarps - 1) / kWarps, kWarps * 32, 0, st>>>(
            nullptr, nullptr, n_items_w, nr, p->ranges, p->pair_item, p->rec, p->desc.width, p->desc.height,
            p->desc.tile_w, p->desc.tile_h, p->TX, p->TY, vb, bg[0], bg[1], bg[2], img, alpha, p->T_final, nc_out,
            p->prof_n_eval, nullptr, nullptr, 0);
    }
    VBM_LAUNCH("raster_fwd");
    record_event(p->prof_ev[1], st);
    note_launches(1);
    return VBM_OK;
}

template <int PPT, int GL>
vbm_status launch_bwd(vbm_plan *p, int vb, int vc, const float bg[3], const float *dimg, const float *dalpha,
                      cudaStream_t st)
{
    const int n_tiles = vc * p->TX * p->TY;
    const int nr = regions_per_tile(p, PPT);
    const int n_items_w = n_tiles * nr;
    record_event(p->prof_ev[2], st);
    if (p->desc.flags & VBM_PLAN_PERSISTENT) {
        // a second backward of the same forward finds the backward's queue
        // counter spent: clear it (the binning clears it for the first)
        if (p->bwd_queue_used) VBM_CUDA(cudaMemsetAsync(p->tile_queue + 1, 0, sizeof(int), st));
        p->bwd_queue_used = true;
        const int grid = persistent_grid(k_raster_bwd<PPT, GL, true>, n_items_w);
        k_raster_bwd<PPT, GL, true><<<grid, kWarps * 32, 0, st>>>(
            p->tile_order, p->tile_queue + 1, n_items_w, nr, p->ranges, p->pair_item, p->rec, p->desc.width, p->desc.height, p->desc.tile_w, p->desc.tile_h, p->TX, p->TY, vb,
            bg[0], bg[1], bg[2], dimg, dalpha, p->T_final, p->n_contrib, p->g_splat, p->tile_queue,
            p->seg_len ? p->seg_units : nullptr, p->ckpt, p->ckpt_base, p->seg_len);
    } else {
        k_raster_bwd<PPT, GL, false><<<(n_items_w + kWarps - 1) / kWarps, kWarps * 32, 0, st>>>(
            nullptr, nullptr, n_items_w, nr, p->ranges, p->pair_item, p->rec, p->desc.width, p->desc.height, p->desc.tile_w, p->desc.tile_h, p->TX, p->TY, vb, bg[0], bg[1],
            bg[2], dimg, dalpha, p->T_final, p->n_contrib, p->g_splat, nullptr, nullptr, nullptr, nullptr, 0);
    }
    VBM_LAUNCH("raster_bwd");
    record_event(p->prof_ev[3], st);
    note_launches(1);
    return VBM_OK;
}

// Dispatch on (pixels per thread, lanes per group).
#define VBM_RASTER_DISPATCH(FN, BWD, ...)                                                             \
    switch (pixels_per_thread(p, BWD) * 64 + group_lanes(p, BWD)) {                                   \
        case 1 * 64 + 4: return FN<1, 4>(__VA_ARGS__);                                                \
        case 1 * 64 + 8: return FN<1, 8>(__VA_ARGS__);                                                \
        case 1 * 64 + 16: return FN<1, 16>(__VA_ARGS__);                                              \
        case 1 * 64 + 32: return FN<1, 32>(__VA_ARGS__);                                              \
        case 2 * 64 + 4: return FN<2, 4>(__VA_ARGS__);                                                \
        case 2 * 64 + 8: return FN<2, 8>(__VA_ARGS__);                                                \
        case 2 * 64 + 16: return FN<2, 16>(__VA_ARGS__);                                              \
        case 2 * 64 + 32: return FN<2, 32>(__VA_ARGS__);                                              \
        case 4 * 64 + 4: return FN<4, 4>(__VA_ARGS__);                                                \
        case 4 * 64 + 8: return FN<4, 8>(__VA_ARGS__);                                                \
        case 4 * 64 + 16: return FN<4, 16>(__VA_ARGS__);                                              \
        case 4 * 64 + 32: return FN<4, 32>(__VA_ARGS__);                                              \
        default: set_error("unsupported pixels-per-thread / group-lanes combination"); return VBM_ERR_ARG; \
    }

}  // namespace

vbm_status raster_fwd(vbm_plan *p, int vb, int vc, const float bg[3], float *img, float *alpha, cudaStream_t st)
{
    VBM_RASTER_DISPATCH(launch_fwd, false, p, vb, vc, bg, img, alpha, st)
}

vbm_status raster_bwd(vbm_plan *p, const float *, int64_t, int vb, int vc, const float bg[3], const float *dimg,
                      const float *dalpha, float *, cudaStream_t st)
{
    // the forward's projection zeroed the splat-gradient records (once the
    // plan has run a backward); otherwise, and for a second backward of the
    // same forward, they are cleared here
    if (!p->g_splat_clear) VBM_CUDA(cudaMemsetAsync(p->g_splat, 0, sizeof(float) * kGradStride * p->last_items, st));
    p->g_splat_clear = false;
    p->bwd_seen = true;
    VBM_RASTER_DISPATCH(launch_bwd, true, p, vb, vc, bg, dimg, dalpha, st)
}

}  // namespace vbm
