// Tile binning with a depth order: per-tile pair counts, ranges, bucket
// placement and a sort of each tile's list.
//
// The order the rasteriser needs is "by tile, then by depth, ties by item
// index".  The projection counts, per tile, the items whose exact tile test
// lists it; an exclusive scan of those counts gives every tile its range of
// the pair array.  Each item then claims one slot per listed tile with an
// atomic decrement of the tile's counter (which the scan set to the range's
// end, and the tile sort clears for the next call) and stores its 64-bit key
// (depth bits << 32 | item) there.  The slots of a tile are filled in arbitrary order, so each tile's
// list is sorted by that key: depth > 0 for every listed item, so the float
// bits order like the depths, and the low word breaks ties by item index.
// The result is unique, so it equals the oracle's (tile, depth, index) sort
// bit for bit however the atomics interleave.
//
// The kernel that walks every tile sorts lists of up to 32 keys with a warp's
// bitonic network in registers and queues the longer ones by size, so that
// each later kernel takes lists of similar cost: up to 256 keys a warp's
// merge sort in shared memory (one warp per list), up to 1024 a 128-thread
// block's, up to 4096 a 512-thread block's; longer lists run the bitonic
// network with its long-distance steps in global memory.  A plan option
// (VBM_PLAN_RADIX_SORT) orders the pairs by device LSD radix sorts instead,
// with the same result.
//
// Compared with sorting all pairs on a (tile | depth) key, nothing is sorted
// globally: the pair array is written once by the placement and once by the
// per-tile sort.  Every kernel runs on a grid fixed by the plan's sizes and
// reads counts from device memory, so a whole step can be captured in a CUDA
// graph without knowing the pair count on the host.
#include <algorithm>

#include "vbm_internal.h"

namespace vbm {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;                        // tiles per thread of a scan chunk
constexpr int kTilesPerChunk = kScanThreads * kScanItems;
constexpr uint64_t kPadKey = ~0ull;

// Longest-list-first order of the tiles for the persistent compositing
// kernels: tiles are grouped by floor(log2(length + 1)), longest group first
// (order within a group is arbitrary; each tile is processed independently).
// A grid-stride kernel after the range scan counts the groups (and claims the
// list segments), and the warp sort places each tile into the order before it
// sorts; lanes of a warp with the same group share one atomic.  The words q hold the two work-queue counters
// (q[0], q[1]), the group sizes (q[2 + g]) and the group cursors (q[34 + g]),
// then the list-segment counters; the first scan kernel zeroes them.
//
// With list segments of length L (seg_len > 0), the counting also gives each tile
// whose list is longer than L ceil(len / L) - 1 checkpoint slots (one per
// segment boundary), plus one for its final per-pixel state when the plan
// stores none (final_slot), and ceil(len / L) backward work units (tile,
// segment), and records the tile's first slot in ckpt_base (-1 for every other
// tile, and for a long tile that finds no free slot, which is then walked
// whole).  Segmented tiles are placed first in the order.  Each segmented tile
// has at least two segments, so the units claimed never exceed twice the slots
// claimed: seg_units holds 2 ckpt_cap entries.
struct TileOrder {
    int *q;              // queue words (NULL: no ordering, non-persistent plans)
    int *order;          // [tiles]
    int seg_len;         // 0: lists are never split
    int final_slot;      // 1 in plans that keep no per-pixel state
    int64_t ckpt_cap;
    int *ckpt_base;      // [tiles] (NULL when seg_len is 0)
    int2 *seg_units;     // [2 ckpt_cap]
};

__device__ __forceinline__ int length_group(int len) { return __clz(len + 1); }   // 31 = length 0; smaller = longer

// Checkpoint slots and backward units of tile t with a list of len entries.
// Returns true if the tile is segmented.
__device__ __forceinline__ bool claim_segments(int len, int t, const TileOrder &o)
{
    int base = -1;
    if (o.seg_len > 0 && len > o.seg_len) {
        const int nseg = (len + o.seg_len - 1) / o.seg_len;
        const int need = nseg - 1 + o.final_slot;
        const int b = atomicAdd(&o.q[kQSegSlots], need);
        if ((int64_t)b + need <= o.ckpt_cap) {
            base = b;
            const int u = atomicAdd(&o.q[kQSegUnits], nseg);
            for (int k = 0; k < nseg; k++) o.seg_units[u + k] = make_int2(t, k);
            atomicAdd(&o.q[kQSegTiles], 1);
        }
    }
    o.ckpt_base[t] = base;
    return base >= 0;
}

// ------------------------------------------------------------ tile ranges

// Sum of the tile counts of each chunk of kTilesPerChunk tiles.
// Also zeroes the queue words of the tile order (q, if not NULL).
__global__ void __launch_bounds__(kScanThreads) k_tile_chunk_sums(const uint32_t *__restrict__ tile_count,
                                                                  int64_t n_tiles, int64_t *__restrict__ chunk_sums,
                                                                  int *__restrict__ q)
{
    if (q && blockIdx.x == 0)
        for (int i = threadIdx.x; i < kTileQueueWords; i += kScanThreads) q[i] = 0;
    __shared__ int64_t warp_sums[kScanThreads / 32];
    const int64_t beg = (int64_t)blockIdx.x * kTilesPerChunk;
    int64_t s = 0;
#pragma unroll
    for (int it = 0; it < kScanItems; it++) {
        const int64_t t = beg + it * kScanThreads + threadIdx.x;
        if (t < n_tiles) s += tile_count[t];
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t tot = 0;
        for (int w = 0; w < kScanThreads / 32; w++) tot += warp_sums[w];
        chunk_sums[blockIdx.x] = tot;
    }
}

// Exclusive scan of the tile counts into ranges [begin, end) ((0, 0) for an
// empty tile); each non-empty tile's counter becomes its range's end, the
// cursor the placement claims slots from.  Each block adds up the sums of the
// chunks before its own and of all chunks.  If the total exceeds the capacity
// every range is empty, the pair count is 0, the counters are cleared and the
// status records the size needed.  Also resets the long-list queue of the
// sort.
__global__ void __launch_bounds__(kScanThreads) k_tile_scan(uint32_t *__restrict__ tile_count, int64_t n_tiles,
                                                            const int64_t *__restrict__ chunk_sums, int chunks,
                                                            int64_t capacity, int2 *__restrict__ ranges,
                                                            int64_t *__restrict__ n_pairs,
                                                            int64_t *__restrict__ status,
                                                            uint32_t *__restrict__ long_count)
{
    __shared__ int64_t red[2][kScanThreads / 32];
    __shared__ int64_t warp_off[kScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t before = 0, total = 0;
    for (int c = threadIdx.x; c < chunks; c += kScanThreads) {
        const int64_t v = chunk_sums[c];
        total += v;
        if (c < (int)blockIdx.x) before += v;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        before += __shfl_xor_sync(0xffffffffu, before, off);
        total += __shfl_xor_sync(0xffffffffu, total, off);
    }
    if (lane == 0) {
        red[0][warp] = before;
        red[1][warp] = total;
    }
    __syncthreads();
    before = total = 0;
    for (int w = 0; w < kScanThreads / 32; w++) {
        before += red[0][w];
        total += red[1][w];
    }
    const bool overflow = total > capacity;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *n_pairs = overflow ? 0 : total;
        long_count[0] = long_count[1] = long_count[2] = 0;
        if (overflow) {
            atomicOr((unsigned long long *)&status[0], (unsigned long long)kStatusCapacity);
            atomicMax((unsigned long long *)&status[1], (unsigned long long)total);
        }
    }
    // thread t scans kScanItems consecutive tiles of the chunk
    const int64_t t0 = (int64_t)blockIdx.x * kTilesPerChunk + (int64_t)threadIdx.x * kScanItems;
    uint32_t c[kScanItems];
    int64_t local = 0;
#pragma unroll
    for (int it = 0; it < kScanItems; it++) {
        c[it] = t0 + it < n_tiles ? tile_count[t0 + it] : 0u;
        local += c[it];
    }
    int64_t incl = local;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) warp_off[warp] = incl;
    __syncthreads();
    int64_t run = before + incl - local;
    for (int w = 0; w < warp; w++) run += warp_off[w];
#pragma unroll
    for (int it = 0; it < kScanItems; it++) {
        const int64_t t = t0 + it;
        if (t >= n_tiles) break;
        if (overflow) {
            ranges[t] = make_int2(0, 0);
            tile_count[t] = 0u;
        } else {
            ranges[t] = c[it] ? make_int2((int)run, (int)(run + c[it])) : make_int2(0, 0);
            if (c[it]) tile_count[t] = (uint32_t)(run + c[it]);   // claim cursor: the range's end
        }
        run += c[it];
    }
}

// Tile counts of each length group and the list-segment claims, one tile per
// thread over a grid-stride loop (segmented tiles are placed ahead of the
// groups); one shared atomic per group among a warp's lanes.  A kernel of its
// own with a full grid: in the scan's few blocks, a thread's consecutive long
// tiles would chain their claims' atomic round trips.
__global__ void __launch_bounds__(kScanThreads) k_tile_group_count(const int2 *__restrict__ ranges, int64_t n_tiles,
                                                                   TileOrder o)
{
    __shared__ int hist[32];
    if (threadIdx.x < 32) hist[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t0 = (int64_t)blockIdx.x * blockDim.x; t0 < n_tiles; t0 += stride) {   // uniform per block
        const int64_t t = t0 + threadIdx.x;
        int g = 32 + lane;                                      // no group: unique per lane
        if (t < n_tiles) {
            const int2 r = ranges[t];
            g = length_group(r.y - r.x);
            if (o.ckpt_base && claim_segments(r.y - r.x, (int)t, o)) g = 32 + lane;
        }
        const uint32_t peers = __match_any_sync(0xffffffffu, g);
        if (g < 32 && lane == __ffs(peers) - 1) atomicAdd(&hist[g], __popc(peers));
    }
    __syncthreads();
    if (threadIdx.x < 32 && hist[threadIdx.x]) atomicAdd(&o.q[2 + threadIdx.x], hist[threadIdx.x]);
}

// ---------------------------------------------------------- placement

// One thread per (view, Gaussian) item, in the projection's grid: the item's
// key goes to one claimed slot of each listed tile (the projection's
// listed-tile word; wide rectangles are tested again with the same code).
// Nothing is placed when the pairs overflowed.
__global__ void k_place_pairs(const int64_t *__restrict__ scene_offset, const int32_t *__restrict__ view_scene,
                              const int64_t *__restrict__ view_item_offset, int vb, const uint4 *__restrict__ place,
                              const SplatRec *__restrict__ rec, int TX, int TY,
                              int tw, int th, int W, int H, uint32_t *__restrict__ tile_count,
                              const int64_t *__restrict__ n_pairs, uint64_t *__restrict__ pair_key)
{
    const int64_t n_total = *n_pairs;
    if (n_total == 0) return;
    const int v = vb + blockIdx.y;
    const int scene = view_scene ? view_scene[v] : 0;
    const int64_t ns = scene_offset[scene + 1] - scene_offset[scene];
    const int64_t gl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t word = 0;
    TileTest t = {};
    uint64_t key = 0;
    if (gl < ns) {                     // every lane stays for the warp-wide placement
        const int64_t item = view_item_offset[v] - view_item_offset[vb] + gl;
        const uint4 pl = place[item];
        word = pl.z;
        if (word) {
            t.rc = place_rect(pl);
            key = ((uint64_t)pl.w << 32) | (uint64_t)(uint32_t)item;
            if (word & kWideRect) {
                const float4 g = rec[item].g, cu = rec[item].cu, x = rec[item].x;
                t = TileTest{g.x, g.y, g.z, g.w, x.x, cu.z, cu.w, x.y, t.rc};
            }
        }
    }
    place_listed(word, t, (uint32_t)blockIdx.y * (uint32_t)(TX * TY), key, TX, tw, th, W, H, n_total, tile_count,
                 pair_key);
}

// ---------------------------------------------------------- tile sort

__device__ __forceinline__ void write_sorted(uint64_t k, int64_t i, uint32_t tile, uint32_t *__restrict__ pair_tile,
                                             uint32_t *__restrict__ pair_item)
{
    pair_item[i] = (uint32_t)k;
    pair_tile[i] = tile;
}

// Bitonic sort, ascending, of a warp's 32 keys (one per lane) through shuffles.
__device__ __forceinline__ uint64_t warp_bitonic32(uint64_t a)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const bool lower = (lane & j) == 0, up = (lane & k) == 0;
            const uint64_t p = __shfl_xor_sync(0xffffffffu, (unsigned long long)a, j);
            const uint64_t lo = a < p ? a : p, hi = a < p ? p : a;
            a = lower == up ? lo : hi;
        }
    }
    return a;
}

// Merge sort of up to G * kMergeE keys by a group of G threads (a warp or a
// block): each thread sorts 8 consecutive keys with Batcher's odd-even merge
// network (19 comparators), then runs of length L = 8, 16, ... are merged
// pairwise, each thread writing 8 consecutive outputs of its pair after a
// binary search for its start on the merge path.  Shared-memory word w is
// stored at w + w / 16, so the 32 lanes' 8-key strides fall in different
// banks.
constexpr int kMergeE = 8;
__host__ __device__ constexpr int padded(int w) { return w + (w >> 4); }

__device__ __forceinline__ void cswap(uint64_t &a, uint64_t &b)
{
    const uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
    a = lo;
    b = hi;
}

__device__ __forceinline__ void sort8(uint64_t (&v)[8])
{
    cswap(v[0], v[1]); cswap(v[2], v[3]); cswap(v[4], v[5]); cswap(v[6], v[7]);
    cswap(v[0], v[2]); cswap(v[1], v[3]); cswap(v[4], v[6]); cswap(v[5], v[7]);
    cswap(v[1], v[2]); cswap(v[5], v[6]);
    cswap(v[0], v[4]); cswap(v[1], v[5]); cswap(v[2], v[6]); cswap(v[3], v[7]);
    cswap(v[2], v[4]); cswap(v[3], v[5]);
    cswap(v[1], v[2]); cswap(v[3], v[4]); cswap(v[5], v[6]);
}

// Outputs [8t, 8t + 8) of the merge of the two sorted runs that contain
// position 8t: [base, base + L) and [base + L, base + 2L), both clipped to the
// first n8 positions (ties: the first run first).
__device__ __forceinline__ void merge_pass(const uint64_t *__restrict__ src, uint64_t *__restrict__ dst, int L, int t,
                                           int n8)
{
    const int o = t * kMergeE;
    const int base = o & ~(2 * L - 1);
    const int d = o - base;
    const uint64_t *A = src, *B = src;
    const int a0 = base, b0 = base + L;
    const int La = min(L, n8 - a0), Lb = max(0, min(L, n8 - b0));
    int lo = max(0, d - Lb), hi = min(d, La);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (A[padded(a0 + mid)] <= B[padded(b0 + d - 1 - mid)]) lo = mid + 1;
        else hi = mid;
    }
    int i = lo, j = d - lo;
    uint64_t a = i < La ? A[padded(a0 + i)] : 0ull, b = j < Lb ? B[padded(b0 + j)] : 0ull;
#pragma unroll
    for (int e = 0; e < kMergeE; e++) {
        const bool ta = j >= Lb || (i < La && a <= b);
        dst[padded(o + e)] = ta ? a : b;
        i += ta;
        j += !ta;
        const int next = ta ? a0 + i : b0 + j;
        const bool more = ta ? i < La : j < Lb;
        const uint64_t v = more ? src[padded(next)] : 0ull;
        a = ta ? v : a;
        b = ta ? b : v;
    }
}

template <bool BLOCK>
__device__ __forceinline__ void group_sync()
{
    if (BLOCK) __syncthreads();
    else __syncwarp();
}

// Sorts keys g[0, n) (n <= G * kMergeE) of a group of G threads (thread t of
// the group) with shared buffers s0, s1 of padded(G * kMergeE) words each;
// returns the buffer that holds the sorted keys, followed by ~0 up to the
// next multiple of kMergeE (runs are clipped there, so a list just above a
// power of two merges no padding).  Ends with a group barrier.
template <int G, bool BLOCK>
__device__ __forceinline__ uint64_t *group_merge_sort(const uint64_t *__restrict__ g, int n, uint64_t *s0,
                                                      uint64_t *s1, int t)
{
    const int n8 = (n + kMergeE - 1) / kMergeE * kMergeE;
    for (int i = t; i < n8; i += G) s1[padded(i)] = i < n ? g[i] : kPadKey;
    group_sync<BLOCK>();
    const int T = n8 / kMergeE;
    if (t < T) {
        uint64_t v[kMergeE];
#pragma unroll
        for (int e = 0; e < kMergeE; e++) v[e] = s1[padded(t * kMergeE + e)];
        sort8(v);
#pragma unroll
        for (int e = 0; e < kMergeE; e++) s0[padded(t * kMergeE + e)] = v[e];
    }
    group_sync<BLOCK>();
    uint64_t *src = s0, *dst = s1;
    for (int L = kMergeE; L < n8; L <<= 1) {
        if (t < T) merge_pass(src, dst, L, t, n8);
        group_sync<BLOCK>();
        uint64_t *x = src;
        src = dst;
        dst = x;
    }
    return src;
}

// Bucket-rank sort of a tile's keys g[0, n) (n <= G * kMergeE) by a block of
// G threads.  The keys' high words are the items' depth bits, which order like
// the depths (all positive), so n / 2 buckets spread linearly over the list's
// range of depth bits give keys of nearby depths; every key is placed into its
// bucket (shared-memory counts, an exclusive scan, a claimed slot) and then
// written at its bucket's start plus the number of smaller keys in its bucket
// (the keys are unique, so the ranks are a permutation).  Returns the buffer
// holding the sorted keys, or nullptr when some bucket holds more than
// kBucketMax keys (depths too clustered for this to pay): the caller then
// merge-sorts.  Buffers: a, b of at least n words, cnt and cur of at least
// max(1, n / 2) words.  Ends with a block barrier.
constexpr int kBucketMax = 64;

template <int G>
__device__ uint64_t *bucket_rank_sort(const uint64_t *__restrict__ g, int n, uint64_t *a, uint64_t *b,
                                      uint32_t *cnt, uint32_t *cur, uint32_t *scratch, int t)
{
    constexpr int E = kMergeE;
    const int nb = max(1, n / 2);
    uint64_t key[E];
    uint32_t lo = 0xffffffffu, hi = 0u;
#pragma unroll
    for (int e = 0; e < E; e++) {
        const int i = t + e * G;
        key[e] = i < n ? g[i] : kPadKey;
        if (i < n) {
            const uint32_t d = (uint32_t)(key[e] >> 32);
            lo = min(lo, d);
            hi = max(hi, d);
        }
    }
    for (int i = t; i < nb; i += G) cnt[i] = 0u;
    if (t == 0) {
        scratch[0] = 0xffffffffu;   // depth-bit minimum
        scratch[1] = 0u;            // maximum
        scratch[2] = 0u;            // largest bucket
    }
    __syncthreads();
    lo = __reduce_min_sync(0xffffffffu, lo);
    hi = __reduce_max_sync(0xffffffffu, hi);
    if ((t & 31) == 0) {
        atomicMin(&scratch[0], lo);
        atomicMax(&scratch[1], hi);
    }
    __syncthreads();
    const uint32_t dmin = scratch[0];
    // monotone in the depth bits: float conversion, a positive scale, truncation
    const float scale = (float)nb / ((float)(scratch[1] - dmin) + 1.0f);
    int bk[E];
#pragma unroll
    for (int e = 0; e < E; e++) {
        bk[e] = -1;
        if (t + e * G < n) {
            bk[e] = min(nb - 1, (int)((float)((uint32_t)(key[e] >> 32) - dmin) * scale));
            atomicAdd(&cnt[bk[e]], 1u);
        }
    }
    __syncthreads();
    // exclusive scan of the bucket counts: each thread a contiguous chunk,
    // then the chunk totals across the block; the largest bucket on the way
    const int per = (nb + G - 1) / G;
    const int c0 = min(nb, t * per), c1 = min(nb, c0 + per);
    uint32_t run = 0u, big = 0u;
    for (int i = c0; i < c1; i++) {
        run += cnt[i];
        big = max(big, cnt[i]);
    }
    big = __reduce_max_sync(0xffffffffu, big);
    if ((t & 31) == 0) atomicMax(&scratch[2], big);
    // block-wide exclusive scan of the per-thread totals (warp scans, then the warp totals)
    const int lane = t & 31, w = t >> 5;
    uint32_t incl = run;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    uint32_t *wsum = scratch + 4;   // [G / 32]
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    if (scratch[2] > (uint32_t)kBucketMax) return nullptr;   // block-uniform: merge sort instead
    uint32_t base = 0u;
    for (int i = 0; i < w; i++) base += wsum[i];
    uint32_t pos = base + incl - run;
    for (int i = c0; i < c1; i++) {
        const uint32_t c = cnt[i];
        cur[i] = pos;
        cnt[i] = pos;          // bucket start (the count is cur - start after the claims)
        pos += c;
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < E; e++)
        if (bk[e] >= 0) a[atomicAdd(&cur[bk[e]], 1u)] = key[e];
    __syncthreads();
#pragma unroll
    for (int e = 0; e < E; e++) {
        if (bk[e] < 0) continue;
        const uint32_t s0 = cnt[bk[e]], s1 = cur[bk[e]];
        uint32_t r = s0;
        for (uint32_t j = s0; j < s1; j++) r += a[j] < key[e];
        b[r] = key[e];
    }
    __syncthreads();
    return b;
}

constexpr int kSortWarps = 8;                                    // warps per block of k_tile_sort_warp
constexpr int kWarpSortMax = 32 * kMergeE;                       // longest list one warp sorts
constexpr int kWarpBufWords = padded(kWarpSortMax);
constexpr int kMidSortThreads = 128;
constexpr int kMidSortMax = kMidSortThreads * kMergeE;           // longest list a 128-thread block sorts
constexpr int kMidBufWords = padded(kMidSortMax);
constexpr int kBlockSortThreads = 512;
constexpr int kBlockSortKeys = kBlockSortThreads * kMergeE;      // longest list sorted in shared memory
constexpr int kBlockBufWords = padded(kBlockSortKeys);
constexpr size_t kBlockSortSmem = 2 * kBlockBufWords * sizeof(uint64_t) +
                                  (kBlockSortKeys + 4 + kBlockSortThreads / 32) * sizeof(uint32_t);

// One warp per tile (grid-stride over the tiles): lists of up to 32 keys are
// sorted in registers; longer ones are queued for k_tile_sort_medium (up to
// kWarpSortMax keys), k_tile_sort_mid (up to kMidSortMax) or k_tile_sort_block,
// so that each of those kernels takes lists of similar cost.  Also clears every tile's counter
// for the next call and, with an ordering (o.q), first places every tile into
// the longest-first order (the scan has counted the groups).  With sort = 0
// (radix-sort ordering) it only clears the counters and places the tiles.
__global__ void __launch_bounds__(kSortWarps * 32) k_tile_sort_warp(const int2 *__restrict__ ranges, int64_t n_tiles,
                                                                    const uint64_t *__restrict__ pair_key,
                                                                    uint32_t *__restrict__ pair_tile,
                                                                    uint32_t *__restrict__ pair_item,
                                                                    uint32_t *__restrict__ tile_count,
                                                                    uint32_t *__restrict__ long_tiles,
                                                                    uint32_t *__restrict__ long_count, TileOrder o,
                                                                    int sort)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (o.q) {                                                  // grid-uniform
        __shared__ int base[32];
        if (threadIdx.x < 32) {
            const int cnt = o.q[2 + threadIdx.x];
            int incl = cnt;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, off);
                if ((int)threadIdx.x >= off) incl += y;
            }
            base[threadIdx.x] = incl - cnt + (o.ckpt_base ? o.q[kQSegTiles] : 0);
        }
        __syncthreads();
        const uint32_t lt_mask = (1u << lane) - 1u;
        const int64_t stride = (int64_t)gridDim.x * blockDim.x;
        for (int64_t t0 = (int64_t)blockIdx.x * blockDim.x; t0 < n_tiles; t0 += stride) {   // uniform per block
            const int64_t t = t0 + threadIdx.x;
            int g = 32 + lane;
            if (t < n_tiles) {
                const int2 r = ranges[t];
                g = length_group(r.y - r.x);
                if (o.ckpt_base && o.ckpt_base[t] >= 0) {
                    o.order[atomicAdd(&o.q[kQSegCursor], 1)] = (int)t;
                    g = 32 + lane;
                }
            }
            const uint32_t peers = __match_any_sync(0xffffffffu, g);
            const int leader = __ffs(peers) - 1;
            int first = 0;
            if (g < 32 && lane == leader) first = atomicAdd(&o.q[34 + g], __popc(peers));
            first = __shfl_sync(0xffffffffu, first, leader);
            if (g < 32) o.order[base[g] + first + __popc(peers & lt_mask)] = (int)t;
        }
    }
    const int64_t warps = (int64_t)gridDim.x * kSortWarps;
    for (int64_t t = (int64_t)blockIdx.x * kSortWarps + w; t < n_tiles; t += warps) {
        const int2 r = ranges[t];
        const int n = r.y - r.x;
        if (lane == 0) tile_count[t] = 0u;
        if (n == 0 || !sort) continue;                          // radix ordering: counters only
        const uint64_t *keys = pair_key + r.x;
        if (n > kWarpSortMax) {
            // queued: lists up to kMidSortMax from the front for k_tile_sort_mid,
            // longer ones from the back for k_tile_sort_block
            if (lane == 0) {
                if (n <= kMidSortMax) long_tiles[atomicAdd(&long_count[0], 1u)] = (uint32_t)t;
                else long_tiles[n_tiles - 1 - atomicAdd(&long_count[1], 1u)] = (uint32_t)t;
            }
        } else if (n <= 32) {
            const uint64_t a = warp_bitonic32(lane < n ? keys[lane] : kPadKey);
            if (lane < n) write_sorted(a, r.x + lane, (uint32_t)t, pair_tile, pair_item);
        } else if (lane == 0) {   // 33 to kWarpSortMax keys: queued for k_tile_sort_medium
            long_tiles[n_tiles + atomicAdd(&long_count[2], 1u)] = (uint32_t)t;
        }
    }
}

// Lists of 33 to kWarpSortMax keys, one warp per list (grid-stride over the
// queue k_tile_sort_warp filled): the warp's merge sort in shared memory.
__global__ void __launch_bounds__(kSortWarps * 32) k_tile_sort_medium(const int2 *__restrict__ ranges,
                                                                      int64_t n_tiles,
                                                                      const uint64_t *__restrict__ pair_key,
                                                                      uint32_t *__restrict__ pair_tile,
                                                                      uint32_t *__restrict__ pair_item,
                                                                      const uint32_t *__restrict__ long_tiles,
                                                                      const uint32_t *__restrict__ long_count)
{
    __shared__ uint64_t buf[kSortWarps][2][kWarpBufWords];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t n_med = long_count[2];
    const uint32_t warps = gridDim.x * kSortWarps;
    for (uint32_t q = blockIdx.x * kSortWarps + w; q < n_med; q += warps) {
        const uint32_t tile = long_tiles[n_tiles + q];
        const int2 r = ranges[tile];
        const int n = r.y - r.x;
        const uint64_t *src = group_merge_sort<32, false>(pair_key + r.x, n, buf[w][0], buf[w][1], lane);
        for (int i = lane; i < n; i += 32) write_sorted(src[padded(i)], r.x + i, tile, pair_tile, pair_item);
        __syncwarp();
    }
}

// Lists of kWarpSortMax + 1 to kMidSortMax keys, one 128-thread block per list
// at a time (grid-stride over the front of the queue): the block's merge sort
// in shared memory, every thread with 8 keys of the padded list at most.
__global__ void __launch_bounds__(kMidSortThreads) k_tile_sort_mid(const int2 *__restrict__ ranges,
                                                                   const uint64_t *__restrict__ pair_key,
                                                                   uint32_t *__restrict__ pair_tile,
                                                                   uint32_t *__restrict__ pair_item,
                                                                   const uint32_t *__restrict__ long_tiles,
                                                                   const uint32_t *__restrict__ long_count)
{
    __shared__ uint64_t buf[2][kMidBufWords];
    __shared__ uint32_t cnt[kMidSortMax / 2], cur[kMidSortMax / 2], scratch[4 + kMidSortThreads / 32];
    const uint32_t n_mid = long_count[0];
    const int t = threadIdx.x;
    for (uint32_t q = blockIdx.x; q < n_mid; q += gridDim.x) {
        const uint32_t tile = long_tiles[q];
        const int2 r = ranges[tile];
        const int n = r.y - r.x;
        const uint64_t *src;
        uint64_t *bs = bucket_rank_sort<kMidSortThreads>(pair_key + r.x, n, buf[0], buf[1], cnt, cur, scratch, t);
        if (bs) {
            for (int i = t; i < n; i += kMidSortThreads) write_sorted(bs[i], r.x + i, tile, pair_tile, pair_item);
            __syncthreads();
            continue;
        }
        src = group_merge_sort<kMidSortThreads, true>(pair_key + r.x, n, buf[0], buf[1], t);
        for (int i = t; i < n; i += kMidSortThreads) write_sorted(src[padded(i)], r.x + i, tile, pair_tile, pair_item);
        __syncthreads();
    }
}

// Ascending compare-exchange of s[i] and s[l] (i < l).
template <typename I>
__device__ __forceinline__ void cex(uint64_t *s, I i, I l)
{
    const uint64_t x = s[i], y = s[l];
    if (y < x) {
        s[i] = y;
        s[l] = x;
    }
}

// Partner pairs of the bitonic network in the form whose comparators all put
// the smaller key first: step (k, j) pairs i with i ^ (k - 1) when j = k / 2
// (the flip) and with i + j otherwise; p enumerates the pairs' lower indices
// (p = q j + r gives i = 2 q j + r = 2 p - r; k and j are powers of two).
template <typename I>
__device__ __forceinline__ void pair_of(I p, I k, I j, I &i, I &l)
{
    i = 2 * p - (p & (j - 1));
    l = j == (k >> 1) ? i ^ (k - 1) : i + j;
}

// The steps of distance j_top, j_top / 2, ..., 1 of a stage whose flip
// distance is larger (every pair is (i, i + j)), on the N0 keys (a power of
// two) in shared memory; block-wide, ends with a barrier.
__device__ void smem_stage_tail(uint64_t *s, int N0, int j_top)
{
    for (int j = j_top; j > 0; j >>= 1) {
        for (int p = threadIdx.x; p < N0 / 2; p += blockDim.x) {
            const int i = 2 * p - (p & (j - 1));
            cex(s, padded(i), padded(i + j));
        }
        __syncthreads();
    }
}

// Sorts the queued long lists, one block per list at a time.  A list of at
// most kBlockSortKeys keys is merge-sorted in shared memory.  A longer one
// (N = its length rounded up to a power of two, positions >= n read as
// +infinity, so comparators that reach them change nothing) runs the bitonic
// network: its chunks of kBlockSortKeys are first merge-sorted (which is what
// the network's first stages produce), then every later stage applies its
// steps of distance >= kBlockSortKeys in global memory and the rest chunk by
// chunk in shared memory.
__global__ void __launch_bounds__(kBlockSortThreads) k_tile_sort_block(const int2 *__restrict__ ranges,
                                                                       uint64_t *__restrict__ pair_key,
                                                                       uint32_t *__restrict__ pair_tile,
                                                                       uint32_t *__restrict__ pair_item,
                                                                       const uint32_t *__restrict__ long_tiles,
                                                                       const uint32_t *__restrict__ long_count,
                                                                       int64_t n_tiles)
{
    extern __shared__ uint64_t smem_keys[];
    uint64_t *s0 = smem_keys, *s1 = smem_keys + kBlockBufWords;
    uint32_t *cnt = reinterpret_cast<uint32_t *>(s1 + kBlockBufWords), *cur = cnt + kBlockSortKeys / 2;
    uint32_t *scratch = cur + kBlockSortKeys / 2;
    const uint32_t n_long = long_count[1];
    const int t = threadIdx.x;
    for (uint32_t q = blockIdx.x; q < n_long; q += gridDim.x) {
        const uint32_t tile = long_tiles[n_tiles - 1 - q];
        const int2 r = ranges[tile];
        const int64_t n = r.y - r.x;
        uint64_t *g = pair_key + r.x;
        if (n <= kBlockSortKeys) {
            uint64_t *bs = bucket_rank_sort<kBlockSortThreads>(g, (int)n, s0, s1, cnt, cur, scratch, t);
            if (bs) {
                for (int i = t; i < n; i += kBlockSortThreads) write_sorted(bs[i], r.x + i, tile, pair_tile, pair_item);
                __syncthreads();
                continue;
            }
            const uint64_t *src = group_merge_sort<kBlockSortThreads, true>(g, (int)n, s0, s1, t);
            for (int i = t; i < n; i += kBlockSortThreads) write_sorted(src[padded(i)], r.x + i, tile, pair_tile, pair_item);
            __syncthreads();
            continue;
        }
        int64_t N = 1;
        while (N < n) N <<= 1;
        const int S = kBlockSortKeys;
        for (int64_t c0 = 0; c0 < n; c0 += S) {
            const int nc = (int)(n - c0 < S ? n - c0 : S);
            const uint64_t *src = group_merge_sort<kBlockSortThreads, true>(g + c0, nc, s0, s1, t);
            for (int i = t; i < nc; i += kBlockSortThreads) g[c0 + i] = src[padded(i)];
            __syncthreads();
        }
        for (int64_t k = 2 * (int64_t)S; k <= N; k <<= 1) {
            for (int64_t j = k >> 1; j >= S; j >>= 1) {
                for (int64_t p = t; p < N / 2; p += kBlockSortThreads) {
                    int64_t i, l;
                    pair_of(p, k, j, i, l);
                    if (l < n) cex(g, i, l);
                }
                __syncthreads();
            }
            for (int64_t c0 = 0; c0 < n; c0 += S) {
                for (int i = t; i < S; i += kBlockSortThreads) s0[padded(i)] = c0 + i < n ? g[c0 + i] : kPadKey;
                __syncthreads();
                smem_stage_tail(s0, S, S >> 1);
                for (int i = t; i < S && c0 + i < n; i += kBlockSortThreads) {
                    if (k == N) write_sorted(s0[padded(i)], r.x + c0 + i, tile, pair_tile, pair_item);
                    else g[c0 + i] = s0[padded(i)];
                }
                __syncthreads();
            }
        }
    }
}

// ------------------------------------------------- radix-sort ordering
//
// VBM_PLAN_RADIX_SORT orders the pairs the way 3D Gaussian Splatting does,
// by a device-wide sort on (tile | depth) keys, split into two stable LSD
// radix sorts on 32-bit keys: the items by their depth bits (ties keep the
// item order), then the pairs, emitted in that depth order, by their tile id
// (ceil(log2 tiles) bits).  Stability carries the (depth, item) order into
// every tile's list, so the lists equal the bucketed per-tile sort's bit for
// bit.  Each radix pass is reduce-then-scan on a fixed grid (per-block digit
// histograms, one block per digit for the offsets, a stable scatter), reading
// the element count from device memory; no block waits on another.

constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kRadixThreads = 256;
constexpr int kRadixWarps = kRadixThreads / 32;
constexpr int kRadixItems = 8;                       // elements per thread per tile
constexpr int kRadixTile = kRadixThreads * kRadixItems;

__device__ __forceinline__ int64_t radix_chunk(int64_t n, int blocks)
{
    const int64_t c = (n + blocks - 1) / blocks;
    return (c + kRadixTile - 1) / kRadixTile * kRadixTile;
}

// Per-block digit histogram of the block's chunk: hist[d * blocks + b], and
// the per-digit totals over all blocks (digit_total, zeroed before).  Equal
// digits within a warp share one shared-memory atomic.
__global__ void __launch_bounds__(kRadixThreads) k_radix_upsweep(const uint32_t *__restrict__ keys,
                                                                 const int64_t *__restrict__ d_n, int shift,
                                                                 uint32_t *__restrict__ hist,
                                                                 uint32_t *__restrict__ digit_total)
{
    __shared__ uint32_t h[kRadix];
    for (int i = threadIdx.x; i < kRadix; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int64_t n = *d_n;
    const int64_t chunk = radix_chunk(n, gridDim.x);
    const int64_t beg = (int64_t)blockIdx.x * chunk;
    const int64_t end = min(n, beg + chunk);
    const int lane = threadIdx.x & 31;
    for (int64_t b = beg; b < end; b += kRadixTile) {       // uniform trip count across the block
        uint32_t d[kRadixItems];
#pragma unroll
        for (int it = 0; it < kRadixItems; it++) {
            const int64_t i = b + it * kRadixThreads + threadIdx.x;
            d[it] = i < end ? (keys[i] >> shift) & (kRadix - 1) : (uint32_t)(kRadix + lane);
        }
#pragma unroll
        for (int it = 0; it < kRadixItems; it++) {
            const uint32_t peers = __match_any_sync(0xffffffffu, d[it]);
            if (d[it] < kRadix && lane == __ffs(peers) - 1) atomicAdd(&h[d[it]], (uint32_t)__popc(peers));
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += blockDim.x) {
        hist[(int64_t)d * gridDim.x + blockIdx.x] = h[d];
        if (h[d]) atomicAdd(&digit_total[d], h[d]);
    }
}

// Exclusive scan of one value per thread over the block; the total goes to
// *total if not NULL.  Ends with a barrier.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t *warp_sums, uint32_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t incl = x;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const uint32_t w = lane < nw ? warp_sums[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, off);
            if (lane >= off) wi += y;
        }
        if (lane < nw) warp_sums[lane] = wi - w;
        if (lane == 31 && total) *total = wi;
    }
    __syncthreads();
    const uint32_t r = warp_sums[warp] + incl - x;
    __syncthreads();
    return r;
}

// Digit-major exclusive offsets, one block per digit d: base(d) = the totals
// of the smaller digits, then a scan of digit d's per-block counts.
__global__ void __launch_bounds__(kRadixThreads) k_radix_offsets(uint32_t *__restrict__ hist,
                                                                 const uint32_t *__restrict__ digit_total,
                                                                 int blocks)
{
    __shared__ uint32_t warp_sums[32];
    __shared__ uint32_t s_base, chunk_total;
    const int d = blockIdx.x;
    uint32_t lower = 0;
    for (int i = threadIdx.x; i < d; i += blockDim.x) lower += digit_total[i];
    (void)block_exclusive_scan(lower, warp_sums, &s_base);
    uint32_t carry = s_base;
    __syncthreads();
    uint32_t *h = hist + (int64_t)d * blocks;
    for (int b0 = 0; b0 < blocks; b0 += blockDim.x) {
        const int b = b0 + threadIdx.x;
        const uint32_t x = b < blocks ? h[b] : 0u;
        const uint32_t ex = block_exclusive_scan(x, warp_sums, &chunk_total);
        if (b < blocks) h[b] = carry + ex;
        __syncthreads();
        carry += chunk_total;
        __syncthreads();
    }
}

// Stable scatter of the block's chunk, one tile of kRadixTile elements at a
// time: within a tile each warp ranks its elements among equal digits
// (earlier iterations of the warp + earlier lanes, from __match_any_sync), the
// tile is exchanged through shared memory into digit order, and written out
// with consecutive threads on consecutive elements of each digit's run.
__global__ void __launch_bounds__(kRadixThreads) k_radix_downsweep(const uint32_t *__restrict__ keys_in,
                                                                   const uint32_t *__restrict__ vals_in,
                                                                   uint32_t *__restrict__ keys_out,
                                                                   uint32_t *__restrict__ vals_out,
                                                                   const int64_t *__restrict__ d_n, int shift,
                                                                   const uint32_t *__restrict__ hist)
{
    static_assert(kRadixThreads == kRadix, "one thread per digit in the per-tile digit scans");
    __shared__ uint32_t run[kRadix];        // global position of the next element of each digit
    __shared__ uint32_t tstart[kRadix];     // first position of each digit in the exchanged tile
    __shared__ uint32_t wcnt[kRadixWarps][kRadix];
    __shared__ uint32_t s_key[kRadixTile];
    __shared__ uint32_t s_val[kRadixTile];
    __shared__ uint32_t warp_sums[32];
    const int64_t n = *d_n;
    const int64_t chunk = radix_chunk(n, gridDim.x);
    const int64_t beg = (int64_t)blockIdx.x * chunk;
    const int64_t end = min(n, beg + chunk);
    if (beg >= end) return;                 // uniform across the block
    const int t = threadIdx.x;
    run[t] = hist[(int64_t)t * gridDim.x + blockIdx.x];
    const int warp = t >> 5, lane = t & 31;
    const uint32_t lt_mask = (1u << lane) - 1u;
    for (int64_t tbase = beg; tbase < end; tbase += kRadixTile) {
#pragma unroll
        for (int w = 0; w < kRadixWarps; w++) wcnt[w][t] = 0;
        __syncthreads();
        uint32_t k[kRadixItems], v[kRadixItems], rank[kRadixItems];
        const int64_t wbase = tbase + (int64_t)warp * 32 * kRadixItems;
#pragma unroll
        for (int it = 0; it < kRadixItems; it++) {
            const int64_t i = wbase + it * 32 + lane;
            const bool valid = i < end;
            k[it] = valid ? keys_in[i] : 0u;
            v[it] = valid ? vals_in[i] : 0u;
        }
#pragma unroll
        for (int it = 0; it < kRadixItems; it++) {
            const int64_t i = wbase + it * 32 + lane;
            const bool valid = i < end;
            const uint32_t d = valid ? (k[it] >> shift) & (kRadix - 1) : (uint32_t)(kRadix + lane);
            const uint32_t peers = __match_any_sync(0xffffffffu, d);
            const uint32_t prior = valid ? wcnt[warp][d] : 0u;
            rank[it] = prior + __popc(peers & lt_mask);
            __syncwarp();
            if (valid && lane == __ffs(peers) - 1) wcnt[warp][d] = prior + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        // thread t = digit t: exclusive offsets over the warps, then over the digits
        uint32_t tot = 0;
#pragma unroll
        for (int w = 0; w < kRadixWarps; w++) {
            const uint32_t c = wcnt[w][t];
            wcnt[w][t] = tot;
            tot += c;
        }
        tstart[t] = block_exclusive_scan(tot, warp_sums, nullptr);
        __syncthreads();
#pragma unroll
        for (int it = 0; it < kRadixItems; it++) {
            const int64_t i = wbase + it * 32 + lane;
            if (i < end) {
                const uint32_t d = (k[it] >> shift) & (kRadix - 1);
                const uint32_t lpos = tstart[d] + wcnt[warp][d] + rank[it];
                s_key[lpos] = k[it];
                s_val[lpos] = v[it];
            }
        }
        __syncthreads();
        const int cnt = (int)min((int64_t)kRadixTile, end - tbase);
        for (int i = t; i < cnt; i += kRadixThreads) {
            const uint32_t key = s_key[i];
            const uint32_t d = (key >> shift) & (kRadix - 1);
            const uint32_t pos = run[d] + (uint32_t)i - tstart[d];
            keys_out[pos] = key;
            vals_out[pos] = s_val[i];
        }
        __syncthreads();
        run[t] += tot;
        __syncthreads();
    }
}

// Item count of the call into a device scalar, and each item's depth key
// (float bits: depth > 0 for every item with tiles, so the bits order like the
// depths; items without tiles sort last) with the item index as value.
__global__ void k_item_keys(int64_t n, const uint4 *__restrict__ place, const uint32_t *__restrict__ touched,
                            uint32_t *__restrict__ key, uint32_t *__restrict__ val, int64_t *__restrict__ d_n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *d_n = n;
    if (i >= n) return;
    key[i] = touched[i] ? place[i].w : 0xffffffffu;
    val[i] = (uint32_t)i;
}

// Exclusive scan of touched[] in the depth order (out[s] = first pair of
// item idx[s], out[n] = the total): per-block sums, one block scanning them,
// then the per-block scans.
constexpr int kGatherItems = 4;

__device__ __forceinline__ int64_t gather_chunk(int64_t n, int blocks)
{
    const int64_t t = kScanThreads * kGatherItems;
    const int64_t c = (n + blocks - 1) / blocks;
    return (c + t - 1) / t * t;
}

__global__ void __launch_bounds__(kScanThreads) k_gather_reduce(const uint32_t *__restrict__ counts,
                                                                const uint32_t *__restrict__ idx, int64_t n,
                                                                int64_t *__restrict__ block_sums)
{
    __shared__ int64_t red[kScanThreads];
    const int64_t chunk = gather_chunk(n, gridDim.x);
    const int64_t beg = (int64_t)blockIdx.x * chunk;
    const int64_t end = min(n, beg + chunk);
    int64_t s = 0;
    for (int64_t i = beg + threadIdx.x; i < end; i += blockDim.x) s += counts[idx[i]];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < (unsigned)off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) block_sums[blockIdx.x] = red[0];
}

// Exclusive scan of the per-block sums (blocks <= 1024) in one block; total at [blocks].
__global__ void __launch_bounds__(1024) k_gather_top(int64_t *__restrict__ block_sums, int blocks)
{
    __shared__ int64_t warp_sums[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t x = (int)threadIdx.x < blocks ? block_sums[threadIdx.x] : 0;
    int64_t incl = x;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int64_t w = warp_sums[lane];
        int64_t wi = w;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, wi, off);
            if (lane >= off) wi += y;
        }
        warp_sums[lane] = wi - w;
        if (lane == 31) block_sums[blocks] = wi;
    }
    __syncthreads();
    if ((int)threadIdx.x < blocks) block_sums[threadIdx.x] = warp_sums[warp] + incl - x;
}

__global__ void __launch_bounds__(kScanThreads) k_gather_down(const uint32_t *__restrict__ counts,
                                                              const uint32_t *__restrict__ idx, int64_t n,
                                                              const int64_t *__restrict__ block_sums,
                                                              int64_t *__restrict__ out)
{
    __shared__ int64_t warp_sums[kScanThreads / 32];
    __shared__ int64_t carry;
    const int64_t chunk = gather_chunk(n, gridDim.x);
    const int64_t beg = (int64_t)blockIdx.x * chunk;
    const int64_t end = min(n, beg + chunk);
    if (threadIdx.x == 0) carry = block_sums[blockIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t tb = beg; tb < end; tb += kScanThreads * kGatherItems) {
        int64_t v[kGatherItems];
        int64_t local = 0;
#pragma unroll
        for (int it = 0; it < kGatherItems; it++) {
            const int64_t i = tb + (int64_t)threadIdx.x * kGatherItems + it;
            v[it] = i < end ? (int64_t)counts[idx[i]] : 0;
            local += v[it];
        }
        int64_t incl = local;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
        }
        if (lane == 31) warp_sums[warp] = incl;
        __syncthreads();
        int64_t wpre = 0, tot = 0;
        for (int w = 0; w < kScanThreads / 32; w++) {
            if (w < warp) wpre += warp_sums[w];
            tot += warp_sums[w];
        }
        int64_t r = carry + wpre + incl - local;
#pragma unroll
        for (int it = 0; it < kGatherItems; it++) {
            const int64_t i = tb + (int64_t)threadIdx.x * kGatherItems + it;
            if (i < end) out[i] = r;
            r += v[it];
        }
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = block_sums[gridDim.x];
}

// Pairs of the items in depth order: item idx[s] owns [offsets[s],
// offsets[s + 1]).  Nothing is emitted when the total exceeds the capacity
// (the tile scan has already reported it).
__global__ void k_emit_pairs(const uint32_t *__restrict__ idx, const int64_t *__restrict__ offsets, int64_t n,
                             const uint4 *__restrict__ place, const SplatRec *__restrict__ rec, const int64_t *__restrict__ view_item_offset, int vb, int vc, int TX, int TY, int tw,
                             int th, int W, int H, int64_t capacity, uint32_t *__restrict__ pair_tile,
                             uint32_t *__restrict__ pair_item)
{
    if (offsets[n] > capacity) return;
    const int64_t base_item = view_item_offset[vb];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // warp-uniform trip count: emit_listed needs every lane of the warp
    for (int64_t s0 = (int64_t)blockIdx.x * blockDim.x; s0 < n; s0 += stride) {
        const int64_t s = s0 + threadIdx.x;
        uint32_t word = 0, item = 0, tile0 = 0;
        int64_t beg = 0;
        TileTest t = {};
        if (s < n && offsets[s + 1] != offsets[s]) {
            beg = offsets[s];
            item = idx[s];
            const uint4 pl = place[item];
            word = pl.z;
            int lo = 0, hi = vc - 1;   // view of the item: last v with offset <= item
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (view_item_offset[vb + mid] - base_item <= (int64_t)item) lo = mid; else hi = mid - 1;
            }
            t.rc = place_rect(pl);
            if (word & kWideRect) {
                const SplatRec r = rec[item];
                t = TileTest{r.g.x, r.g.y, r.g.z, r.g.w, r.x.x, r.cu.z, r.cu.w, r.x.y, t.rc};
            }
            tile0 = (uint32_t)lo * (uint32_t)(TX * TY);
        }
        emit_listed(word, t, tile0, item, beg, TX, tw, th, W, H, pair_tile, pair_item);
    }
}

int ceil_log2(int64_t x)
{
    int b = 0;
    while ((int64_t(1) << b) < x) b++;
    return b;
}

}  // namespace

int bin_chunks(int64_t n_tiles) { return (int)std::max<int64_t>(1, (n_tiles + kTilesPerChunk - 1) / kTilesPerChunk); }

int radix_blocks() { return num_sms() * 4; }
int scan_blocks() { return std::min(1024, num_sms() * 4); }
size_t radix_hist_words(int blocks) { return (size_t)kRadix * blocks + kRadix; }

namespace {

// Stable LSD radix sort of (keys, vals) on their low `bits` key bits, 8 bits
// a pass, between the two buffers; returns the buffer holding the result.
// The grid is fixed by n_max (graph capture); the count is read from d_n.
vbm_status radix_sort(uint32_t *keys[2], uint32_t *vals[2], const int64_t *d_n, int64_t n_max, int bits,
                      const vbm_plan *p, int *result, cudaStream_t st)
{
    int cur = 0;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(p->radix_blocks,
                                                                   (n_max + kRadixTile - 1) / kRadixTile));
    for (int shift = 0; shift < bits; shift += kRadixBits) {
        VBM_CUDA(cudaMemsetAsync(p->radix_total, 0, kRadix * sizeof(uint32_t), st));
        k_radix_upsweep<<<blocks, kRadixThreads, 0, st>>>(keys[cur], d_n, shift, p->radix_hist, p->radix_total);
        VBM_LAUNCH("radix_upsweep");
        k_radix_offsets<<<kRadix, kRadixThreads, 0, st>>>(p->radix_hist, p->radix_total, blocks);
        VBM_LAUNCH("radix_offsets");
        k_radix_downsweep<<<blocks, kRadixThreads, 0, st>>>(keys[cur], vals[cur], keys[1 - cur], vals[1 - cur], d_n,
                                                            shift, p->radix_hist);
        VBM_LAUNCH("radix_downsweep");
        note_launches(3);
        cur = 1 - cur;
    }
    *result = cur;
    return VBM_OK;
}

// Radix-sort ordering of the pairs (VBM_PLAN_RADIX_SORT): the items by depth,
// their pairs emitted in that order, then the pairs stably by tile.  The
// ranges come from the tile scan (the same counts); the result lands in
// pair_tile / pair_item, with the bucketed path's key buffer as the second
// buffer of the pair sort.
vbm_status radix_order(vbm_plan *p, int vb, int vc, int64_t n_tiles, cudaStream_t st)
{
    const int64_t n_items = p->view_item_offset[vb + vc] - p->view_item_offset[vb];
    if (n_items == 0) return VBM_OK;
    k_item_keys<<<(unsigned)((n_items + 255) / 256), 256, 0, st>>>(n_items, p->place, p->touched, p->item_key[0],
                                                                    p->item_val[0], p->d_n_items);
    VBM_LAUNCH("item_keys");
    note_launches(1);
    int a = 0;
    vbm_status s = radix_sort(p->item_key, p->item_val, p->d_n_items, n_items, 32, p, &a, st);
    if (s != VBM_OK) return s;
    k_gather_reduce<<<p->scan_blocks, kScanThreads, 0, st>>>(p->touched, p->item_val[a], n_items, p->scan_sums);
    VBM_LAUNCH("gather_reduce");
    k_gather_top<<<1, 1024, 0, st>>>(p->scan_sums, p->scan_blocks);
    VBM_LAUNCH("gather_top");
    k_gather_down<<<p->scan_blocks, kScanThreads, 0, st>>>(p->touched, p->item_val[a], n_items, p->scan_sums,
                                                            p->item_offset);
    VBM_LAUNCH("gather_down");
    note_launches(3);
    // emit into the buffer from which an even number of tile passes ends in pair_tile / pair_item
    const int64_t cap = p->desc.pair_capacity;
    uint32_t *tiles[2] = {p->pair_tile, reinterpret_cast<uint32_t *>(p->pair_key)};
    uint32_t *items[2] = {p->pair_item, reinterpret_cast<uint32_t *>(p->pair_key) + cap};
    const int tile_bits = ceil_log2(n_tiles);
    const int passes = (tile_bits + kRadixBits - 1) / kRadixBits;
    const int first = passes & 1;
    k_emit_pairs<<<num_sms() * 4, 256, 0, st>>>(p->item_val[a], p->item_offset, n_items, p->place, p->rec,
                                                 p->d_view_item_offset, vb, vc, p->TX,
                                                 p->TY, p->desc.tile_w, p->desc.tile_h, p->desc.width, p->desc.height,
                                                 cap, tiles[first], items[first]);
    VBM_LAUNCH("emit_pairs");
    note_launches(1);
    uint32_t *tk[2] = {tiles[first], tiles[1 - first]};
    uint32_t *tv[2] = {items[first], items[1 - first]};
    int r = 0;
    s = radix_sort(tk, tv, p->d_n_pairs, cap, tile_bits, p, &r, st);
    if (s != VBM_OK) return s;
    if (tk[r] != p->pair_tile) {   // cannot happen: the emission buffer was chosen for this
        set_error("radix ordering ended in the scratch buffer");
        return VBM_ERR_CUDA;
    }
    return VBM_OK;
}

}  // namespace

cudaError_t binning_setup()
{
    return cudaFuncSetAttribute(k_tile_sort_block, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBlockSortSmem);
}

vbm_status binning(vbm_plan *p, int vb, int vc, cudaStream_t st)
{
    const int64_t n_tiles = (int64_t)vc * p->TX * p->TY;
    const BinScratch &b = p->bin_scratch;
    const int chunks = bin_chunks(n_tiles);
    // 1. ranges from the per-tile counts of the projection
    TileOrder o{};
    if (p->desc.flags & VBM_PLAN_PERSISTENT) {
        o.q = p->tile_queue;
        o.order = p->tile_order;
        o.seg_len = p->seg_len;
        o.final_slot = p->T_final ? 0 : 1;
        o.ckpt_cap = p->ckpt_cap;
        o.ckpt_base = p->seg_len ? p->ckpt_base : nullptr;
        o.seg_units = p->seg_units;
    }
    k_tile_chunk_sums<<<chunks, kScanThreads, 0, st>>>(p->tile_count, n_tiles, b.chunk_sums, o.q);
    VBM_LAUNCH("tile_chunk_sums");
    k_tile_scan<<<chunks, kScanThreads, 0, st>>>(p->tile_count, n_tiles, b.chunk_sums, chunks,
                                                 p->desc.pair_capacity, p->ranges, p->d_n_pairs, p->d_status,
                                                 b.long_count);
    VBM_LAUNCH("tile_scan");
    note_launches(2);
    if (o.q) {
        const int og = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)num_sms() * 4,
                                                                   (n_tiles + kScanThreads - 1) / kScanThreads));
        k_tile_group_count<<<og, kScanThreads, 0, st>>>(p->ranges, n_tiles, o);
        VBM_LAUNCH("tile_group_count");
        note_launches(1);
    }
    const bool radix = (p->desc.flags & VBM_PLAN_RADIX_SORT) != 0;
    if (radix) {
        vbm_status s = radix_order(p, vb, vc, n_tiles, st);
        if (s != VBM_OK) return s;
    }
    // 2. every item's key into a slot of each listed tile
    if (!radix && p->max_scene > 0) {
        dim3 grid((unsigned)((p->max_scene + 255) / 256), (unsigned)vc);
        k_place_pairs<<<grid, 256, 0, st>>>(p->d_scene_offset, p->desc.n_scenes > 1 ? p->d_view_scene : nullptr,
                                            p->d_view_item_offset, vb, p->place, p->rec, p->TX, p->TY,
                                            p->desc.tile_w, p->desc.tile_h,
                                            p->desc.width, p->desc.height, p->tile_count, p->d_n_pairs, p->pair_key);
        VBM_LAUNCH("place_pairs");
        note_launches(1);
    }
    // 3. each tile's list sorted by (depth, item)
    // one wave of blocks (more would leave a partial second wave on a few SMs)
    static int sort_per_sm = 0;
    if (sort_per_sm == 0) {
        VBM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&sort_per_sm, k_tile_sort_warp, kSortWarps * 32, 0));
        sort_per_sm = std::max(sort_per_sm, 1);
    }
    const int sw = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)num_sms() * sort_per_sm,
                                                               (n_tiles + kSortWarps - 1) / kSortWarps));
    k_tile_sort_warp<<<sw, kSortWarps * 32, 0, st>>>(p->ranges, n_tiles, p->pair_key, p->pair_tile, p->pair_item,
                                                     p->tile_count, b.long_tiles, b.long_count, o, radix ? 0 : 1);
    VBM_LAUNCH("tile_sort_warp");
    note_launches(1);
    if (!radix) {
        static int medium_per_sm = 0;
        if (medium_per_sm == 0) {
            VBM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&medium_per_sm, k_tile_sort_medium,
                                                                   kSortWarps * 32, 0));
            medium_per_sm = std::max(medium_per_sm, 1);
        }
        k_tile_sort_medium<<<num_sms() * medium_per_sm, kSortWarps * 32, 0, st>>>(
            p->ranges, n_tiles, p->pair_key, p->pair_tile, p->pair_item, b.long_tiles, b.long_count);
        VBM_LAUNCH("tile_sort_medium");
        note_launches(1);
        k_tile_sort_mid<<<num_sms() * 8, kMidSortThreads, 0, st>>>(p->ranges, p->pair_key, p->pair_tile,
                                                                    p->pair_item, b.long_tiles, b.long_count);
        VBM_LAUNCH("tile_sort_mid");
        k_tile_sort_block<<<num_sms() * 2, kBlockSortThreads, kBlockSortSmem, st>>>(
            p->ranges, p->pair_key, p->pair_tile, p->pair_item, b.long_tiles, b.long_count, n_tiles);
        VBM_LAUNCH("tile_sort_block");
        note_launches(2);
    }
    return VBM_OK;
}

}  // namespace vbm
