// Internal declarations shared by the translation units of libvbm.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <climits>
#include <map>
#include <string>
#include <vector>

#include "vbm.h"

namespace vbm {

// Splatting constants (3D Gaussian Splatting conventions, Sec. 4.4 defers
// the fine-tuning loss to that method).
constexpr float kFrustumGuard = 0.15f;  // clamp x/z, y/z to the image +15% per side
constexpr float kDilation = 0.3f;       // added to the 2D covariance diagonal
constexpr float kEigFloor = 0.1f;       // lambda_max = mid + sqrt(max(0.1, mid^2 - det))
constexpr float kRadiusSigmas = 3.0f;   // r = ceil(3 sqrt(lambda_max))
constexpr float kAlphaMax = 0.99f;
constexpr float kAlphaMin = 1.0f / 255.0f;
// Natural-log margin of the compositing kernels' culling tests (far above the
// rounding of the quantities compared).
constexpr float kCullMargin = 1e-3f;
// Floats per item of the splat-gradient records: du dv dA dB dC dopacity dr dg db, padding.
constexpr int kGradStride = 12;

// A projected splat as the binning and compositing kernels read it: one
// aligned 64-byte line per (view, Gaussian) item, so that a list entry costs
// one contiguous 64-byte read (two sectors) whatever its position in memory.
//   g  = u, v, conic A, conic B        c = r, g, b, opacity
//   cu = half-widths of the alpha >= 1/255 box (x, y), B / C, B / A
//   x  = conic C, tau = 2 (ln(255 o) + kCullMargin), camera depth, unused
struct __align__(64) SplatRec {
    float4 g, c, cu, x;
};
static_assert(sizeof(SplatRec) == 64, "one 64-byte line per splat");
// The last word of a SplatRec (x.w) holds the splat radius in pixels (int32 bits).

// Per-item placement record (uint4) written by the projection: the tile
// rectangle [x0, x1) x [y0, y1) as x0 | x1 << 16 and y0 | y1 << 16, the
// listed-tile word (listed_tiles) and the camera depth's float bits, so that
// the pair placement reads one 16-byte load per item.  Plans have at most
// kMaxTilesPerAxis tiles along each axis, so every coordinate fits 16 bits.
constexpr int kMaxTilesPerAxis = 65535;
constexpr int kProfileEvents = 7;       // timing events a plan can record (vbm_plan_set_profile)

// Adam step fused into the projection backward (vbm_raster_bwd_adam): the
// first n columns of P, M, V ([14][stride], updated in place), the device
// step counter (already incremented for this step), per-row-group learning
// rates, and the optional non-finite gradient counter.
struct AdamArgs {
    float *P = nullptr, *M = nullptr, *V = nullptr;
    const int32_t *step = nullptr;
    int64_t n = 0;
    float lr[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    float beta1 = 0.f, beta2 = 0.f, eps = 0.f;
    uint32_t *nonfinite = nullptr;
};

#ifdef __CUDACC__
// Binning tile test: smallest q = A dx^2 + 2 B dx dy + C dy^2 (dx = x - u,
// dy = y - v) over the rectangle [x0, x1] x [y0, y1] of a tile's pixel
// centres: 0 if (u, v) lies inside; else the minimum of a convex quadratic
// over a box lies on an edge whose half-plane excludes the centre (at an
// interior point of an edge the level set through it is tangent to the edge,
// with the centre inside, on the far side; at a corner a line through the
// corner separates the box from that level set), so at most one vertical
// edge (x0 if u < x0, x1 if u > x1) and one horizontal edge are evaluated,
// each by its 1D minimiser (dy = -bc dx, dx = -ba dy with bc = B / C,
// ba = B / A) clamped to the edge.  A tile is listed for a splat when this is
// <= tau = 2 (ln(255 o) + kCullMargin): alpha = o e^(-q/2) >= 1/255 needs
// q <= 2 ln(255 o), so a pixel of an unlisted tile would skip the splat.
// Every operation is an explicitly rounded float32 operation in a fixed order
// (no contraction), so the decision is reproducible bit for bit.
__device__ __forceinline__ float tile_min_q(float u, float v, float A, float B, float C, float bc, float ba,
                                            float x0, float x1, float y0, float y1)
{
    const bool left = u < x0, right = u > x1, below = v < y0, above = v > y1;
    if (!(left || right || below || above)) return 0.f;
    const float inf = __int_as_float(0x7f800000);
    const float B2 = __fmul_rn(2.f, B);
    const float dx = __fsub_rn(left ? x0 : x1, u);
    const float dy = __fsub_rn(fminf(fmaxf(__fsub_rn(v, __fmul_rn(bc, dx)), y0), y1), v);
    const float qv = __fadd_rn(__fadd_rn(__fmul_rn(__fmul_rn(A, dx), dx), __fmul_rn(__fmul_rn(B2, dx), dy)),
                               __fmul_rn(__fmul_rn(C, dy), dy));
    const float ey = __fsub_rn(below ? y0 : y1, v);
    const float ex = __fsub_rn(fminf(fmaxf(__fsub_rn(u, __fmul_rn(ba, ey)), x0), x1), u);
    const float qh = __fadd_rn(__fadd_rn(__fmul_rn(__fmul_rn(A, ex), ex), __fmul_rn(__fmul_rn(B2, ex), ey)),
                               __fmul_rn(__fmul_rn(C, ey), ey));
    return fminf(left || right ? qv : inf, below || above ? qh : inf);
}

// Is tile (tx, ty) of a tw x th grid over a W x H image listed for the splat?
__device__ __forceinline__ bool tile_listed(float u, float v, float A, float B, float C, float bc, float ba,
                                            float tau, int tx, int ty, int tw, int th, int W, int H)
{
    const float x0 = __fadd_rn((float)(tx * tw), 0.5f), x1 = __fsub_rn((float)min(tx * tw + tw, W), 0.5f);
    const float y0 = __fadd_rn((float)(ty * th), 0.5f), y1 = __fsub_rn((float)min(ty * th + th, H), 0.5f);
    return tile_min_q(u, v, A, B, C, bc, ba, x0, x1, y0, y1) <= tau;
}

// One Adam update of a scalar (p, m, v in place; Sec. 5.2 trains with Adam);
// false when g is not finite (nothing is changed).  Every rounding is
// explicit, so the separate Adam kernels and the backward fused with Adam
// give the same bits.
__device__ __forceinline__ bool adam_elem(float &p, float &m, float &v, float g, float lr, float beta1,
                                          float beta2, float eps, float bc1, float bc2)
{
    if (!isfinite(g)) return false;
    m = __fmaf_rn(beta1, m, __fmul_rn(1.f - beta1, g));
    v = __fmaf_rn(beta2, v, __fmul_rn(__fmul_rn(1.f - beta2, g), g));
    const float mhat = __fdiv_rn(m, bc1);
    const float vhat = __fdiv_rn(v, bc2);
    p = __fsub_rn(p, __fdiv_rn(__fmul_rn(lr, mhat), __fadd_rn(__fsqrt_rn(vhat), eps)));
    return true;
}

// Learning rate of parameter row `row`: mean, log-scale, quaternion, opacity, colour.
__device__ __forceinline__ float adam_row_lr(int row, float lr0, float lr1, float lr2, float lr3, float lr4)
{
    return row < 3 ? lr0 : row < 6 ? lr1 : row < 10 ? lr2 : row < 11 ? lr3 : lr4;
}

// Adam's bias corrections 1 - beta^t for step t.
__device__ __forceinline__ float2 adam_bias_corrections(int t, float beta1, float beta2)
{
    return make_float2(1.f - powf(beta1, (float)t), 1.f - powf(beta2, (float)t));
}

// A splat's tile-test record and its radius rectangle (tiles [x, z) x [y, w)).
struct TileTest {
    float u, v, A, B, C, bc, ba, tau;
    int4 rc;
};

__device__ __forceinline__ uint4 pack_place(int4 rc, uint32_t word, float depth)
{
    return make_uint4((uint32_t)rc.x | (uint32_t)rc.z << 16, (uint32_t)rc.y | (uint32_t)rc.w << 16, word,
                      __float_as_uint(depth));
}

__device__ __forceinline__ int4 place_rect(uint4 pl)
{
    return make_int4((int)(pl.x & 0xffffu), (int)(pl.y & 0xffffu), (int)(pl.x >> 16), (int)(pl.y >> 16));
}

// Rectangles of up to this many tiles are tested by their own lane; larger
// ones by the whole warp, 32 tiles at a time (a few large splats would
// otherwise hold their warp for the length of a serial loop).
constexpr int kSerialTiles = 8;

__device__ __forceinline__ TileTest shfl_test(const TileTest &t, int src)
{
    TileTest r;
    r.u = __shfl_sync(0xffffffffu, t.u, src);
    r.v = __shfl_sync(0xffffffffu, t.v, src);
    r.A = __shfl_sync(0xffffffffu, t.A, src);
    r.B = __shfl_sync(0xffffffffu, t.B, src);
    r.C = __shfl_sync(0xffffffffu, t.C, src);
    r.bc = __shfl_sync(0xffffffffu, t.bc, src);
    r.ba = __shfl_sync(0xffffffffu, t.ba, src);
    r.tau = __shfl_sync(0xffffffffu, t.tau, src);
    r.rc.x = __shfl_sync(0xffffffffu, t.rc.x, src);
    r.rc.y = __shfl_sync(0xffffffffu, t.rc.y, src);
    r.rc.z = __shfl_sync(0xffffffffu, t.rc.z, src);
    r.rc.w = __shfl_sync(0xffffffffu, t.rc.w, src);
    return r;
}

__device__ __forceinline__ bool listed_at(const TileTest &t, int col, int row, int tw, int th, int W, int H)
{
    return tile_listed(t.u, t.v, t.A, t.B, t.C, t.bc, t.ba, t.tau, t.rc.x + col, t.rc.y + row, tw, th, W, H);
}

__device__ __forceinline__ uint32_t tile_id_at(const TileTest &t, int col, int row, uint32_t tile0, int TX)
{
    return tile0 + (uint32_t)((t.rc.y + row) * TX + t.rc.x + col);
}

// Row-major position k of a rectangle with `cols` columns as (column, row).
// Below 2^21 positions by a float reciprocal: (k + 1/2) / cols lies at least
// 1 / (2 cols) from an integer, far more than the product's rounding error.
__device__ __forceinline__ int2 rect_pos(int k, int cols, float inv_cols, int area)
{
    const int row = area < (1 << 21) ? (int)(((float)k + 0.5f) * inv_cols) : k / cols;
    return make_int2(k - row * cols, row);
}

// Listed tiles of this lane's rectangle, as one word: 0 when none (or
// !valid); for a rectangle of at most kSerialTiles tiles, bit k set when its
// k-th tile (row-major) is listed; for a larger one, kWideRect (its tiles are
// tested again, by the whole warp, where they are needed).  With tile_count,
// adds one to the counter of every listed tile (tile ids tile0 + row-major
// index in a TX-wide grid).  All 32 lanes of the warp must call it.
constexpr uint32_t kWideRect = 1u << 31;

__device__ __forceinline__ uint32_t listed_tiles(bool valid, const TileTest &t, int tw, int th, int W, int H,
                                                 uint32_t *__restrict__ tile_count, uint32_t tile0, int TX,
                                                 uint32_t *n_listed = nullptr)
{
    const int cols = t.rc.z - t.rc.x;
    const int area = valid ? cols * (t.rc.w - t.rc.y) : 0;
    uint32_t word = 0;
    if (area > 0 && area <= kSerialTiles) {
        int k = 0;
        for (int row = 0; row < t.rc.w - t.rc.y; row++)
            for (int col = 0; col < cols; col++, k++) word |= listed_at(t, col, row, tw, th, W, H) ? 1u << k : 0u;
    }
    // counts of the small rectangles: one atomic per distinct tile among the
    // warp's lanes at each rectangle position (neighbouring items share tiles)
    const int span = __reduce_max_sync(0xffffffffu, word ? 32 - __clz(word) : 0);
    const int lane = threadIdx.x & 31;
    int col = 0, row = 0;
#pragma unroll
    for (int k = 0; k < kSerialTiles; k++) {
        if (k >= span) break;
        const bool on = (word >> k) & 1u;
        const uint32_t id = on ? tile_id_at(t, col, row, tile0, TX) : 0xffffffffu;
        const uint32_t peers = __match_any_sync(0xffffffffu, id);
        if (on && lane == __ffs(peers) - 1) atomicAdd(&tile_count[id], (uint32_t)__popc(peers));
        if (++col == cols) {
            col = 0;
            row++;
        }
    }
    for (uint32_t big = __ballot_sync(0xffffffffu, area > kSerialTiles); big; big &= big - 1) {
        const int src = __ffs(big) - 1;
        const TileTest b = shfl_test(t, src);
        const uint32_t b_tile0 = __shfl_sync(0xffffffffu, tile0, src);
        const int b_cols = b.rc.z - b.rc.x;
        const int a = b_cols * (b.rc.w - b.rc.y);
        const float inv_cols = 1.0f / (float)b_cols;
        uint32_t cnt = 0;
        for (int k0 = 0; k0 < a; k0 += 32) {
            const int k = k0 + lane;
            const int2 pos = rect_pos(k, b_cols, inv_cols, a);
            const bool ok = k < a && listed_at(b, pos.x, pos.y, tw, th, W, H);
            if (ok) atomicAdd(&tile_count[tile_id_at(b, pos.x, pos.y, b_tile0, TX)], 1u);
            cnt += __popc(__ballot_sync(0xffffffffu, ok));
        }
        if (lane == src && cnt) word = kWideRect;
        if (lane == src && n_listed) *n_listed = cnt;
    }
    if (n_listed && !(word & kWideRect)) *n_listed = __popc(word);
    return word;
}

// Bucket placement: for every listed tile of this lane's rectangle (the word
// listed_tiles returned; a wide rectangle's tiles are tested again with the
// same code), claim a slot of that tile's range and store the key there.  The
// tile's counter holds the end of its unclaimed part of the pair array (the
// scan sets it to the range's end), so a claim is one atomic decrement that
// returns the slot directly.  Order within a tile is arbitrary: a sort by key
// follows.  A slot outside [0, n_total) (impossible while the counts and the
// claims take the same decisions) stores nothing.  All 32 lanes must call it;
// t needs only its rectangle unless the word is kWideRect.
__device__ __forceinline__ void place_listed(uint32_t word, const TileTest &t, uint32_t tile0, uint64_t key, int TX,
                                             int tw, int th, int W, int H, int64_t n_total,
                                             uint32_t *__restrict__ tile_count, uint64_t *__restrict__ pair_key)
{
    // small rectangles: lanes claiming the same tile at the same rectangle
    // position share one atomic (the leader takes the group's slots and each
    // lane its rank among them); every claim is issued before the first store
    // depends on one
    const uint32_t small = (word & kWideRect) ? 0u : word;
    const int span = __reduce_max_sync(0xffffffffu, small ? 32 - __clz(small) : 0);
    const int lane = threadIdx.x & 31;
    const int cols = t.rc.z - t.rc.x;
    uint32_t tid[kSerialTiles], peer[kSerialTiles], old[kSerialTiles];
    int col = 0, row = 0;
#pragma unroll
    for (int k = 0; k < kSerialTiles; k++) {
        old[k] = 0u;
        if (k >= span) continue;
        const bool on = (small >> k) & 1u;
        tid[k] = on ? tile_id_at(t, col, row, tile0, TX) : 0xffffffffu;
        peer[k] = __match_any_sync(0xffffffffu, tid[k]);
        if (on && lane == __ffs(peer[k]) - 1) old[k] = atomicSub(&tile_count[tid[k]], (uint32_t)__popc(peer[k]));
        if (++col == cols) {
            col = 0;
            row++;
        }
    }
#pragma unroll
    for (int k = 0; k < kSerialTiles; k++) {
        if (k >= span) break;
        if (!((small >> k) & 1u)) continue;
        const uint32_t o = __shfl_sync(peer[k], old[k], __ffs(peer[k]) - 1);
        const int64_t slot = (int64_t)o - __popc(peer[k]) + __popc(peer[k] & ((1u << lane) - 1u));
        if (slot >= 0 && slot < n_total) pair_key[slot] = key;
    }
    for (uint32_t big = __ballot_sync(0xffffffffu, (word & kWideRect) != 0); big; big &= big - 1) {
        const int src = __ffs(big) - 1;
        const TileTest b = shfl_test(t, src);
        const uint32_t b_tile0 = __shfl_sync(0xffffffffu, tile0, src);
        const uint64_t b_key = __shfl_sync(0xffffffffu, (unsigned long long)key, src);
        const int b_cols = b.rc.z - b.rc.x;
        const int a = b_cols * (b.rc.w - b.rc.y);
        const float inv_cols = 1.0f / (float)b_cols;
        for (int k0 = 0; k0 < a; k0 += 32) {
            const int k = k0 + lane;
            const int2 pos = rect_pos(k, b_cols, inv_cols, a);
            if (k < a && listed_at(b, pos.x, pos.y, tw, th, W, H)) {
                const uint32_t id = tile_id_at(b, pos.x, pos.y, b_tile0, TX);
                const int64_t slot = (int64_t)atomicSub(&tile_count[id], 1u) - 1;
                if (slot >= 0 && slot < n_total) pair_key[slot] = b_key;
            }
        }
    }
}

// Pair emission in a given order (radix-sort ordering): the lane's item owns
// pair slots [beg, beg + its listed-tile count) and writes one (tile, item)
// pair per listed tile of its rectangle, row-major (a wide rectangle's tiles
// are tested again, by the whole warp, with the same code).  All 32 lanes must
// call it; word = 0 for a lane without an item.
__device__ __forceinline__ void emit_listed(uint32_t word, const TileTest &t, uint32_t tile0, uint32_t item,
                                            int64_t beg, int TX, int tw, int th, int W, int H,
                                            uint32_t *__restrict__ pair_tile, uint32_t *__restrict__ pair_item)
{
    const int lane = threadIdx.x & 31;
    if (word && !(word & kWideRect)) {
        const int cols = t.rc.z - t.rc.x;
        int64_t o = beg;
        int col = 0, row = 0;
        for (int k = 0; k < kSerialTiles; k++) {
            if ((word >> k) & 1u) {
                pair_tile[o] = tile_id_at(t, col, row, tile0, TX);
                pair_item[o] = item;
                o++;
            }
            if (++col == cols) {
                col = 0;
                row++;
            }
        }
    }
    for (uint32_t big = __ballot_sync(0xffffffffu, (word & kWideRect) != 0); big; big &= big - 1) {
        const int src = __ffs(big) - 1;
        const TileTest b = shfl_test(t, src);
        const uint32_t b_tile0 = __shfl_sync(0xffffffffu, tile0, src);
        const uint32_t b_item = __shfl_sync(0xffffffffu, item, src);
        int64_t run = (int64_t)__shfl_sync(0xffffffffu, (long long)beg, src);
        const int b_cols = b.rc.z - b.rc.x;
        const int a = b_cols * (b.rc.w - b.rc.y);
        const float inv_cols = 1.0f / (float)b_cols;
        for (int k0 = 0; k0 < a; k0 += 32) {
            const int k = k0 + lane;
            const int2 pos = rect_pos(k, b_cols, inv_cols, a);
            const bool ok = k < a && listed_at(b, pos.x, pos.y, tw, th, W, H);
            const uint32_t bal = __ballot_sync(0xffffffffu, ok);
            if (ok) {
                const int64_t o = run + __popc(bal & ((1u << lane) - 1u));
                pair_tile[o] = tile_id_at(b, pos.x, pos.y, b_tile0, TX);
                pair_item[o] = b_item;
            }
            run += __popc(bal);
        }
    }
}
#endif
constexpr float kTMin = 1e-4f;
constexpr float kCoordClamp = 1e7f;

// Device status word bits of a plan.
constexpr uint32_t kStatusCapacity = 1u;

void set_error(const std::string &msg);
vbm_status cuda_fail(cudaError_t e, const char *what);

#define VBM_CUDA(call)                                                  \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return ::vbm::cuda_fail(e_, #call);      \
    } while (0)

#define VBM_LAUNCH(what)                                                \
    do {                                                                \
        cudaError_t e_ = cudaGetLastError();                            \
        if (e_ != cudaSuccess) return ::vbm::cuda_fail(e_, what);       \
    } while (0)

#define VBM_ARG(cond, msg)                                              \
    do {                                                                \
        if (!(cond)) { ::vbm::set_error(msg); return VBM_ERR_ARG; }     \
    } while (0)

int num_sms();

// Host-side count of kernel launches (diagnostics).
void note_launches(int n);

// Record an event on a stream; under stream capture as an external node so the
// caller can read its time after the graph replays.
void record_event(cudaEvent_t ev, cudaStream_t st);

// Wavelet filter bank {tap index: coefficient} in the periodised convention
// a[k] = sum_n ht[n] x[2k+n], d[k] = sum_n gt[n] x[2k+1+n],
// x[m] = sum_k h[m-2k] a[k] + g[m-2k-1] d[k].  wavelet 0 = bior4.4, 1 = Haar.
struct FilterBank {
    std::map<int, double> ht, gt, h, g;
};
FilterBank make_filters(int wavelet);

// ---------------------------------------------------------------- binning
// Work-queue counters of the compositing kernels (2), tile-group sizes and
// cursors of the longest-first order (32 + 32), then the list-segment
// counters: backward segment units, segmented tiles, claimed checkpoint
// slots, and the placement cursor of the segmented tiles.
constexpr int kTileQueueWords = 2 + 32 + 32 + 4;
constexpr int kQSegUnits = 66, kQSegTiles = 67, kQSegSlots = 68, kQSegCursor = 69;

// List segments (persistent plans): a tile whose list is longer than the
// segment length L is walked by the backward as ceil(len / L) independent
// work units of L entries.  The forward stores, per pixel of such a tile, the
// transmittance and the colour still to come at each segment boundary (one
// float4 checkpoint slot of tile_w x tile_h records per boundary); plans that
// keep no per-pixel state (recompute) also store the tile's final state
// (transmittance, last contributor) in one more slot, so the backward replays
// only the short lists.  Checkpoint memory is bounded; tiles that find no
// free slot are walked whole.
constexpr int kDefaultSegmentLen = 256;
constexpr int64_t kCheckpointPairsPerItem = 2;
constexpr int64_t kCheckpointBytes = 1ll << 30;

// Scratch of the binning: per-chunk sums of the tile counts and the lists of
// tiles too long for one warp's sort (mid-size from the front, the longest
// from the back).
struct BinScratch {
    int64_t *chunk_sums = nullptr;  // [chunks]
    int chunks = 0;                 // ceil(max tiles / tiles per chunk)
    uint32_t *long_tiles = nullptr; // [2 max tiles]: mid and longest lists, then medium ones
    uint32_t *long_count = nullptr; // [3] queued lists for the mid, the block and the medium sort
};
int bin_chunks(int64_t n_tiles);
cudaError_t binning_setup();   // once per plan, before any capture: kernel attributes
int radix_blocks();            // blocks of the radix-sort kernels
int scan_blocks();             // blocks of the item scan (<= 1024)
size_t radix_hist_words(int blocks);

}  // namespace vbm

// ------------------------------------------------------------------ plan
struct vbm_plan {
    vbm_plan_desc desc{};
    std::vector<int64_t> scene_offset;      // host copy
    std::vector<int32_t> view_scene;        // host copy
    std::vector<int64_t> view_item_offset;  // [V + 1] items of view v start at this offset
    int TX = 0, TY = 0;
    int64_t max_scene = 0;                  // largest scene
    int64_t n_gauss = 0;                    // scene_offset[n_scenes]
    int64_t items_cap = 0;                  // view_item_offset[V]

    // device copies of the batch description
    int64_t *d_scene_offset = nullptr;
    int32_t *d_view_scene = nullptr;
    int64_t *d_view_item_offset = nullptr;
    int32_t *d_scene_view_ptr = nullptr;    // CSR scene -> views
    int32_t *d_scene_views = nullptr;

    // per item
    vbm::SplatRec *rec = nullptr;            // [items] the projected splat, one 64-byte line
    uint4 *place = nullptr;                  // [items] tile rectangle, listed-tile word, depth (placement record)
    float *g_splat = nullptr;               // [items][kGradStride]
    bool g_splat_clear = false;             // host: zeroed by the last forward, no backward since
    bool bwd_seen = false;                  // host: a backward has run on this plan
    bool bwd_queue_used = false;            // host: a persistent backward has taken its work queue since
                                            // the last binning zeroed the counters

    // pairs
    uint64_t *pair_key = nullptr;            // [pairs] (depth bits << 32 | item), bucketed by tile
    uint32_t *pair_tile = nullptr;           // [pairs] sorted
    uint32_t *pair_item = nullptr;           // [pairs] sorted
    uint32_t *tile_count = nullptr;          // [V * TX * TY] listed pairs per tile, then the placement's
                                             // claim cursor (zero between calls)
    int2 *ranges = nullptr;                  // [V * TX * TY]
    int *tile_order = nullptr;               // [V * TX * TY] longest list first (persistent mode)
    int *tile_queue = nullptr;               // [kTileQueueWords]: work-queue counters (forward, backward),
                                             // then tile-group sizes and cursors of the ordering
    int seg_len = 0;                         // list segment length L (0: lists are never split)
    int64_t ckpt_cap = 0;                    // checkpoint slots
    float4 *ckpt = nullptr;                  // [ckpt_cap][tile_w * tile_h] (T, colour to come) at boundaries,
                                             // then (recompute plans) (T_final, last contributor bits, 0, 0)
    int *ckpt_base = nullptr;                // [V * TX * TY] first slot of a segmented tile, else -1
    int2 *seg_units = nullptr;               // [2 * ckpt_cap] (tile, segment) backward work units

    // radix-sort ordering (VBM_PLAN_RADIX_SORT)
    uint32_t *touched = nullptr;             // [items] listed tiles per item
    uint32_t *item_key[2] = {nullptr, nullptr};   // [items] depth bits, double buffer
    uint32_t *item_val[2] = {nullptr, nullptr};   // [items] item index, double buffer
    int64_t *item_offset = nullptr;          // [items + 1] first pair of each item in depth order
    int64_t *d_n_items = nullptr;            // items of the call (device scalar)
    uint32_t *radix_hist = nullptr;          // [256 * radix_blocks + 256]
    uint32_t *radix_total = nullptr;         // [256]
    int64_t *scan_sums = nullptr;            // [scan_blocks + 1]
    int radix_blocks = 0, scan_blocks = 0;

    // per pixel
    float *T_final = nullptr;
    int32_t *n_contrib = nullptr;

    // scratch + counters
    vbm::BinScratch bin_scratch;
    int64_t *d_n_pairs = nullptr;            // pairs of the last call
    int64_t *d_status = nullptr;             // [0] status bits, [1] max pairs needed

    // profiling hooks
    cudaEvent_t prof_ev[vbm::kProfileEvents] = {};
    int32_t *prof_n_eval = nullptr;
    int32_t *prof_n_contrib = nullptr;       // contributor counts of recompute-mode forwards (profiling)

    // last forward call
    int32_t last_view_begin = -1, last_view_count = 0;
    int64_t last_items = 0;
    std::vector<void *> allocations;
};

namespace vbm {
vbm_status preprocess_fwd(vbm_plan *p, const float *params, int64_t stride, const vbm_camera *cams, int vb, int vc,
                          cudaStream_t st);
vbm_status binning(vbm_plan *p, int vb, int vc, cudaStream_t st);
vbm_status raster_fwd(vbm_plan *p, int vb, int vc, const float bg[3], float *img, float *alpha, cudaStream_t st);
vbm_status raster_bwd(vbm_plan *p, const float *params, int64_t stride, int vb, int vc, const float bg[3],
                      const float *dimg, const float *dalpha, float *grad, cudaStream_t st);
vbm_status preprocess_bwd(vbm_plan *p, const float *params, int64_t stride, const vbm_camera *cams, int vb, int vc,
                          float *grad, int accumulate, cudaStream_t st, const AdamArgs *adam = nullptr);
vbm_status adam_step_inc(int32_t *step, cudaStream_t st);
}  // namespace vbm
