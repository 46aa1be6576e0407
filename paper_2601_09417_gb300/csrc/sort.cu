// Tile binning with a depth order: scans, a stable LSD radix sort, pair
// emission and tile ranges.
//
// The order the rasteriser needs is "by tile, then by depth, ties by item
// index".  Instead of sorting every (tile, Gaussian) pair on a 64-bit
// (tile | depth) key, the items are first sorted by their 32-bit depth key
// (N x V elements), the pairs are then emitted in that depth order, and a
// stable sort on the tile id alone (ceil(log2 #tiles) bits, usually two 8-bit
// passes) groups them by tile.  Stability carries the depth order (and the
// item-index tie break of the first stable sort) into every tile's list, so
// the result equals the 64-bit sort while the large pair array is sorted on
// ~16 key bits instead of ~45 and each pair is 8 bytes instead of 12.
//
// Every kernel here runs on a fixed grid (a multiple of the SM count) and
// reads element counts from device memory, so a whole step can be captured
// in a CUDA graph without knowing the pair count on the host.  No kernel
// waits on another block: the radix sort is reduce-then-scan (upsweep
// histograms, one scan block, downsweep scatter).
#include <algorithm>

#include "vbm_internal.h"

namespace vbm {
namespace {

constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 8;                      // elements per thread per tile
constexpr int kSortTile = kSortThreads * kSortItems;

__device__ __forceinline__ int64_t chunk_of(int64_t n, int blocks)
{
    int64_t c = (n + blocks - 1) / blocks;
    return (c + kSortTile - 1) / kSortTile * kSortTile;
}

// Per-block digit histogram of keys in the block's chunk: hist[d * blocks + b],
// and the per-digit totals over all blocks (digit_total, zeroed before).
// Equal digits within a warp are counted with one shared-memory atomic
// (__match_any_sync groups them), so keys that share their high bits do not
// serialise on one counter.
__global__ void __launch_bounds__(kSortThreads) k_radix_upsweep(const uint32_t *__restrict__ keys,
                                                                const int64_t *__restrict__ d_n, int shift,
                                                                uint32_t *__restrict__ hist,
                                                                uint32_t *__restrict__ digit_total)
{
    __shared__ uint32_t h[kRadix];
    for (int i = threadIdx.x; i < kRadix; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int64_t n = *d_n;
    const int64_t chunk = chunk_of(n, gridDim.x);
    const int64_t beg = (int64_t)blockIdx.x * chunk;
    const int64_t end = min(n, beg + chunk);
    const int lane = threadIdx.x & 31;
    for (int64_t b = beg; b < end; b += kSortTile) {       // uniform trip count across the block
        uint32_t d[kSortItems];
#pragma unroll
        for (int it = 0; it < kSortItems; it++) {           // all loads of the tile first
            const int64_t i = b + it * kSortThreads + threadIdx.x;
            d[it] = i < end ? (keys[i] >> shift) & (kRadix - 1) : (uint32_t)(kRadix + lane);
        }
#pragma unroll
        for (int it = 0; it < kSortItems; it++) {
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
        uint32_t w = lane < nw ? warp_sums[lane] : 0u;
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

// Digit-major exclusive offsets, one block per digit d: base(d) = sum of the
// totals of the smaller digits, then a scan of digit d's per-block counts.
__global__ void __launch_bounds__(kSortThreads) k_radix_offsets(uint32_t *__restrict__ hist,
                                                                const uint32_t *__restrict__ digit_total, int blocks)
{
    __shared__ uint32_t warp_sums[32];
    __shared__ uint32_t s_base;
    const int d = blockIdx.x;
    uint32_t lower = 0;
    for (int i = threadIdx.x; i < d; i += blockDim.x) lower += digit_total[i];
    const uint32_t dummy = block_exclusive_scan(lower, warp_sums, &s_base);
    (void)dummy;
    __syncthreads();
    uint32_t carry = s_base;
    __syncthreads();
    uint32_t *h = hist + (int64_t)d * blocks;
    for (int b0 = 0; b0 < blocks; b0 += blockDim.x) {
        const int b = b0 + threadIdx.x;
        const uint32_t x = b < blocks ? h[b] : 0u;
        __shared__ uint32_t chunk_total;
        const uint32_t ex = block_exclusive_scan(x, warp_sums, &chunk_total);
        if (b < blocks) h[b] = carry + ex;
        __syncthreads();
        carry += chunk_total;
        __syncthreads();
    }
}

// Stable scatter of the block's chunk, one tile of kSortTile elements at a
// time.  Ranking: within a tile, warp w owns elements [w * 32 * kSortItems,
// (w + 1) * 32 * kSortItems) and walks them 32 at a time; the rank of an
// element among equal digits of the warp is (earlier iterations of this warp)
// + (earlier lanes of this iteration, from __match_any_sync).  The tile is
// then exchanged through shared memory into digit order (digit start in the
// tile + elements of that digit in earlier warps + rank), and written out
// with consecutive threads on consecutive elements, so each digit's run of
// the tile goes to global memory as contiguous stores.
__global__ void __launch_bounds__(kSortThreads) k_radix_downsweep(const uint32_t *__restrict__ keys_in,
                                                                  const uint32_t *__restrict__ vals_in,
                                                                  uint32_t *__restrict__ keys_out,
                                                                  uint32_t *__restrict__ vals_out,
                                                                  const int64_t *__restrict__ d_n, int shift,
                                                                  const uint32_t *__restrict__ hist)
{
    static_assert(kSortThreads == kRadix, "one thread per digit in the per-tile digit scans");
    __shared__ uint32_t run[kRadix];        // global position of the next element of each digit
    __shared__ uint32_t tstart[kRadix];     // first position of each digit in the exchanged tile
    __shared__ uint32_t wcnt[kSortWarps][kRadix];
    __shared__ uint32_t s_key[kSortTile];
    __shared__ uint32_t s_val[kSortTile];
    __shared__ uint32_t warp_sums[32];
    const int64_t n = *d_n;
    const int64_t chunk = chunk_of(n, gridDim.x);
    const int64_t beg = (int64_t)blockIdx.x * chunk;
    const int64_t end = min(n, beg + chunk);
    if (beg >= end) return;                 // uniform across the block
    const int t = threadIdx.x;
    run[t] = hist[(int64_t)t * gridDim.x + blockIdx.x];
    const int warp = t >> 5, lane = t & 31;
    const uint32_t lt_mask = (1u << lane) - 1u;
    for (int64_t tbase = beg; tbase < end; tbase += kSortTile) {
#pragma unroll
        for (int w = 0; w < kSortWarps; w++) wcnt[w][t] = 0;
        __syncthreads();
        uint32_t k[kSortItems], v[kSortItems], rank[kSortItems];
        const int64_t wbase = tbase + (int64_t)warp * 32 * kSortItems;
#pragma unroll
        for (int it = 0; it < kSortItems; it++) {
            const int64_t i = wbase + it * 32 + lane;
            const bool valid = i < end;
            k[it] = valid ? keys_in[i] : 0u;
            v[it] = valid ? vals_in[i] : 0u;
        }
#pragma unroll
        for (int it = 0; it < kSortItems; it++) {
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
        for (int w = 0; w < kSortWarps; w++) {
            const uint32_t c = wcnt[w][t];
            wcnt[w][t] = tot;
            tot += c;
        }
        tstart[t] = block_exclusive_scan(tot, warp_sums, nullptr);
        __syncthreads();
#pragma unroll
        for (int it = 0; it < kSortItems; it++) {
            const int64_t i = wbase + it * 32 + lane;
            if (i < end) {
                const uint32_t d = (k[it] >> shift) & (kRadix - 1);
                const uint32_t lpos = tstart[d] + wcnt[warp][d] + rank[it];
                s_key[lpos] = k[it];
                s_val[lpos] = v[it];
            }
        }
        __syncthreads();
        const int cnt = (int)min((int64_t)kSortTile, end - tbase);
        for (int i = t; i < cnt; i += kSortThreads) {
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

// ------------------------------------------------------------ gather scan

constexpr int kScanThreads = 256;
constexpr int kScanItems = 4;

__device__ __forceinline__ int64_t scan_chunk(int64_t n, int blocks)
{
    const int64_t t = kScanThreads * kScanItems;
    int64_t c = (n + blocks - 1) / blocks;
    return (c + t - 1) / t * t;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t *__restrict__ counts,
                                                              const uint32_t *__restrict__ idx, int64_t n,
                                                              int64_t *__restrict__ block_sums)
{
    __shared__ int64_t red[kScanThreads];
    const int64_t chunk = scan_chunk(n, gridDim.x);
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
__global__ void __launch_bounds__(1024) k_scan_top(int64_t *__restrict__ block_sums, int blocks)
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

__global__ void __launch_bounds__(kScanThreads) k_scan_down(const uint32_t *__restrict__ counts,
                                                            const uint32_t *__restrict__ idx, int64_t n,
                                                            const int64_t *__restrict__ block_sums,
                                                            int64_t *__restrict__ out)
{
    __shared__ int64_t warp_sums[kScanThreads / 32];
    __shared__ int64_t carry;
    const int64_t chunk = scan_chunk(n, gridDim.x);
    const int64_t beg = (int64_t)blockIdx.x * chunk;
    const int64_t end = min(n, beg + chunk);
    if (threadIdx.x == 0) carry = block_sums[blockIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t tb = beg; tb < end; tb += kScanThreads * kScanItems) {
        int64_t v[kScanItems];
        int64_t local = 0;
#pragma unroll
        for (int it = 0; it < kScanItems; it++) {
            const int64_t i = tb + (int64_t)threadIdx.x * kScanItems + it;
            v[it] = i < end ? (int64_t)counts[idx[i]] : 0;
            local += v[it];
        }
        int64_t incl = local;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += y;
        }
        if (lane == 31) warp_sums[warp] = incl;
        __syncthreads();
        int64_t wpre = 0, tot = 0;
        for (int w = 0; w < kScanThreads / 32; w++) {
            if (w < warp) wpre += warp_sums[w];
            tot += warp_sums[w];
        }
        int64_t run = carry + wpre + incl - local;
#pragma unroll
        for (int it = 0; it < kScanItems; it++) {
            const int64_t i = tb + (int64_t)threadIdx.x * kScanItems + it;
            if (i < end) out[i] = run;
            run += v[it];
        }
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = block_sums[gridDim.x];
}

// ------------------------------------------------------------- emission

__global__ void k_set_i64(int64_t *dst, int64_t value)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *dst = value;
}

// Pairs for the items in depth order: item sorted[s] owns [offsets[s],
// offsets[s+1]) and writes one (tile, item) pair per listed tile of its
// rectangle (the tile test preprocess counted with), row-major.  If the
// total exceeds the capacity nothing is emitted, the pair count is set to 0
// and the plan's status records the required size.
__global__ void k_emit_pairs(const uint32_t *__restrict__ sorted, const int64_t *__restrict__ offsets, int64_t n,
                             const int4 *__restrict__ rect, const float4 *__restrict__ geo,
                             const float *__restrict__ conic_c, const float4 *__restrict__ cull,
                             const float *__restrict__ tau, const int64_t *__restrict__ view_item_offset, int vb,
                             int vc, int TX, int TY, int tw, int th, int W, int H, int64_t capacity,
                             uint32_t *__restrict__ pair_tile, uint32_t *__restrict__ pair_item,
                             int64_t *__restrict__ n_pairs, int64_t *__restrict__ status)
{
    const int64_t total = offsets[n];
    const bool overflow = total > capacity;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *n_pairs = overflow ? 0 : total;
        if (overflow) {
            atomicOr((unsigned long long *)&status[0], (unsigned long long)kStatusCapacity);
            atomicMax((unsigned long long *)&status[1], (unsigned long long)total);
        }
    }
    if (overflow) return;
    const int64_t base_item = view_item_offset[vb];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // warp-uniform trip count: emit_listed needs every lane of the warp
    for (int64_t s0 = (int64_t)blockIdx.x * blockDim.x; s0 < n; s0 += stride) {
        const int64_t s = s0 + threadIdx.x;
        bool has = false;
        TileTest t = {};
        uint32_t item = 0, tile0 = 0;
        int64_t beg = 0;
        if (s < n) {
            beg = offsets[s];
            has = offsets[s + 1] != beg;
        }
        if (has) {
            item = sorted[s];
            int lo = 0, hi = vc - 1;   // view of the item: last v with offset <= item
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (view_item_offset[vb + mid] - base_item <= (int64_t)item) lo = mid; else hi = mid - 1;
            }
            const float4 g = geo[item], cu = cull[item];
            t = TileTest{g.x, g.y, g.z, g.w, conic_c[item], cu.z, cu.w, tau[item], rect[item]};
            tile0 = (uint32_t)lo * (uint32_t)(TX * TY);
        }
        emit_listed(has, t, tile0, item, beg, TX, tw, th, W, H, pair_tile, pair_item);
    }
}

__global__ void k_tile_ranges(const uint32_t *__restrict__ tile, const int64_t *__restrict__ n_pairs,
                              int2 *__restrict__ ranges)
{
    const int64_t n = *n_pairs;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t t = tile[i];
        if (i == 0 || tile[i - 1] != t) ranges[t].x = (int)i;
        if (i == n - 1 || tile[i + 1] != t) ranges[t].y = (int)(i + 1);
    }
}

// Longest-list-first order of the tiles for the persistent compositing
// kernels: tiles are grouped by floor(log2(length + 1)), longest group first
// (order within a group is arbitrary; each tile is processed independently).
// Two grid-stride kernels over the tiles: group sizes, then placement.  Lanes
// of a warp with the same group share one atomic.  The scratch q holds the two
// work-queue counters (q[0], q[1]), the group sizes (q[2 + g]) and the group
// cursors (q[34 + g]); it is zeroed before the first kernel.
constexpr int kOrderThreads = 256;

__device__ __forceinline__ int tile_group(const int2 *__restrict__ ranges, int t, int n_tiles, int lane)
{
    if (t >= n_tiles) return 32 + lane;                 // no group: unique per lane
    const int2 r = ranges[t];
    return __clz(r.y - r.x + 1);                        // 31 = length 0; smaller = longer
}

__global__ void __launch_bounds__(kOrderThreads) k_tile_group_count(const int2 *__restrict__ ranges, int n_tiles,
                                                                    int *__restrict__ q)
{
    __shared__ int hist[32];
    if (threadIdx.x < 32) hist[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int stride = gridDim.x * kOrderThreads;
    for (int t0 = blockIdx.x * kOrderThreads; t0 < n_tiles; t0 += stride) {   // uniform per block
        const int g = tile_group(ranges, t0 + (int)threadIdx.x, n_tiles, lane);
        const uint32_t peers = __match_any_sync(0xffffffffu, g);
        if (g < 32 && lane == __ffs(peers) - 1) atomicAdd(&hist[g], __popc(peers));
    }
    __syncthreads();
    if (threadIdx.x < 32 && hist[threadIdx.x]) atomicAdd(&q[2 + threadIdx.x], hist[threadIdx.x]);
}

__global__ void __launch_bounds__(kOrderThreads) k_tile_group_place(const int2 *__restrict__ ranges, int n_tiles,
                                                                    int *__restrict__ q, int *__restrict__ order)
{
    __shared__ int base[32];
    if (threadIdx.x < 32) {
        const int c = q[2 + threadIdx.x];
        int incl = c;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, off);
            if ((int)threadIdx.x >= off) incl += y;
        }
        base[threadIdx.x] = incl - c;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const int stride = gridDim.x * kOrderThreads;
    for (int t0 = blockIdx.x * kOrderThreads; t0 < n_tiles; t0 += stride) {
        const int t = t0 + (int)threadIdx.x;
        const int g = tile_group(ranges, t, n_tiles, lane);
        const uint32_t peers = __match_any_sync(0xffffffffu, g);
        const int leader = __ffs(peers) - 1;
        int first = 0;
        if (g < 32 && lane == leader) first = atomicAdd(&q[34 + g], __popc(peers));
        first = __shfl_sync(0xffffffffu, first, leader);
        if (g < 32) order[base[g] + first + __popc(peers & lt_mask)] = t;
    }
}

int ceil_log2(int64_t x)
{
    int b = 0;
    while ((int64_t(1) << b) < x) b++;
    return b;
}

}  // namespace

size_t radix_sort_hist_words(int blocks) { return (size_t)kRadix * blocks + kRadix; }

int radix_sort_pairs(uint32_t *keys[2], uint32_t *vals[2], const int64_t *d_n, int64_t n_max, int bits,
                     const SortScratch &s, cudaStream_t st)
{
    int cur = 0;
    if (n_max <= 0) return cur;
    // fixed grid for the largest count this call can see (graph capture), at
    // most s.blocks; with fewer elements the trailing blocks have empty chunks
    const int blocks = (int)std::min<int64_t>(s.blocks, (n_max + kSortTile - 1) / kSortTile);
    for (int shift = 0; shift < bits; shift += kRadixBits) {
        cudaMemsetAsync(s.digit_total, 0, kRadix * sizeof(uint32_t), st);
        k_radix_upsweep<<<blocks, kSortThreads, 0, st>>>(keys[cur], d_n, shift, s.hist, s.digit_total);
        k_radix_offsets<<<kRadix, kSortThreads, 0, st>>>(s.hist, s.digit_total, blocks);
        k_radix_downsweep<<<blocks, kSortThreads, 0, st>>>(keys[cur], vals[cur], keys[1 - cur], vals[1 - cur], d_n,
                                                           shift, s.hist);
        cur = 1 - cur;
        note_launches(3);
    }
    return cur;
}

void gather_scan(const uint32_t *counts, const uint32_t *idx, int64_t n, int64_t *out, const ScanScratch &s,
                 cudaStream_t st)
{
    k_scan_reduce<<<s.blocks, kScanThreads, 0, st>>>(counts, idx, n, s.block_sums);
    k_scan_top<<<1, 1024, 0, st>>>(s.block_sums, s.blocks);
    k_scan_down<<<s.blocks, kScanThreads, 0, st>>>(counts, idx, n, s.block_sums, out);
    note_launches(3);
}

vbm_status binning(vbm_plan *p, int vb, int vc, cudaStream_t st)
{
    const int64_t n_items = p->view_item_offset[vb + vc] - p->view_item_offset[vb];
    const int64_t n_tiles = (int64_t)vc * p->TX * p->TY;
    k_set_i64<<<1, 32, 0, st>>>(p->d_n_items, n_items);
    note_launches(1);
    // 1. depth order of the items (stable: ties keep the item order)
    const int a = radix_sort_pairs(p->keyA, p->valA, p->d_n_items, n_items, 32, p->sort_scratch, st);
    // 2. pair offsets in depth order
    gather_scan(p->touched, p->valA[a], n_items, p->offsets, p->scan_scratch, st);
    // 3. emit pairs
    const int grid = num_sms() * 4;
    k_emit_pairs<<<grid, 256, 0, st>>>(p->valA[a], p->offsets, n_items, p->rect, p->geo, p->conic_c, p->cull,
                                       p->tau, p->d_view_item_offset, vb, vc, p->TX, p->TY, p->desc.tile_w,
                                       p->desc.tile_h, p->desc.width, p->desc.height, p->desc.pair_capacity,
                                       p->pair_tile[0], p->pair_item[0], p->d_n_pairs, p->d_status);
    VBM_LAUNCH("emit_pairs");
    note_launches(1);
    // 4. stable sort of the pairs by tile
    p->pair_buf = radix_sort_pairs(p->pair_tile, p->pair_item, p->d_n_pairs, p->desc.pair_capacity,
                                   ceil_log2(n_tiles), p->sort_scratch, st);
    // 5. tile ranges
    VBM_CUDA(cudaMemsetAsync(p->ranges, 0, sizeof(int2) * n_tiles, st));
    k_tile_ranges<<<grid, 256, 0, st>>>(p->pair_tile[p->pair_buf], p->d_n_pairs, p->ranges);
    VBM_LAUNCH("tile_ranges");
    note_launches(1);
    if (p->desc.flags & VBM_PLAN_PERSISTENT) {
        VBM_CUDA(cudaMemsetAsync(p->tile_queue, 0, kTileQueueWords * sizeof(int), st));
        const int64_t og_need = (n_tiles + kOrderThreads - 1) / kOrderThreads;
        const int og = (int)std::max<int64_t>(1, std::min<int64_t>(num_sms() * 2, og_need));
        k_tile_group_count<<<og, kOrderThreads, 0, st>>>(p->ranges, (int)n_tiles, p->tile_queue);
        VBM_LAUNCH("tile_group_count");
        k_tile_group_place<<<og, kOrderThreads, 0, st>>>(p->ranges, (int)n_tiles, p->tile_queue, p->tile_order);
        VBM_LAUNCH("tile_group_place");
        note_launches(2);
    }
    return VBM_OK;
}

}  // namespace vbm
