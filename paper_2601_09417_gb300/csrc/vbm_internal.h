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

// ---------------------------------------------------------------- sorting
// Stable LSD radix sort of (uint32 key, uint32 value) pairs over the low
// `bits` bits of the key; the element count is read from d_n on the device.
// Results end in (keys[0], vals[0]) or (keys[1], vals[1]): the returned index.
constexpr int kTileQueueWords = 2 + 32 + 32;

struct SortScratch {
    uint32_t *hist = nullptr;          // radix * blocks counters
    uint32_t *digit_total = nullptr;   // radix counters (inside the same allocation)
    int blocks = 0;                    // largest sort grid (hist has radix x blocks counters)
};
size_t radix_sort_hist_words(int blocks);
int radix_sort_pairs(uint32_t *keys[2], uint32_t *vals[2], const int64_t *d_n, int64_t n_max, int bits,
                     const SortScratch &s, cudaStream_t st);

// Exclusive scan of uint32 counts gathered through an index array:
// out[i] = sum_{j<i} counts[idx[j]], out[n] = total (int64).
struct ScanScratch {
    int64_t *block_sums = nullptr;  // blocks + 1
    int blocks = 0;
};
void gather_scan(const uint32_t *counts, const uint32_t *idx, int64_t n, int64_t *out, const ScanScratch &s,
                 cudaStream_t st);

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
    float4 *geo = nullptr;
    float4 *col = nullptr;
    float *conic_c = nullptr;
    float4 *cull = nullptr;                  // [items] half-widths of the alpha >= 1/255 box, B / C, B / A
    float *depth = nullptr;
    int4 *rect = nullptr;
    int32_t *radius = nullptr;
    uint32_t *touched = nullptr;
    uint32_t *keyA[2] = {nullptr, nullptr};
    uint32_t *valA[2] = {nullptr, nullptr};
    int64_t *offsets = nullptr;             // [items + 1]
    float *g_splat = nullptr;               // [items][kGradStride]

    // pairs
    uint32_t *pair_tile[2] = {nullptr, nullptr};
    uint32_t *pair_item[2] = {nullptr, nullptr};
    int pair_buf = 0;                        // which buffer holds the sorted pairs
    int2 *ranges = nullptr;                  // [V * TX * TY]
    int *tile_order = nullptr;               // [V * TX * TY] longest list first (persistent mode)
    int *tile_queue = nullptr;               // [kTileQueueWords]: work-queue counters (forward, backward),
                                             // then tile-group sizes and cursors of the ordering

    // per pixel
    float *T_final = nullptr;
    int32_t *n_contrib = nullptr;

    // scratch + counters
    vbm::SortScratch sort_scratch;
    vbm::ScanScratch scan_scratch;
    int64_t *d_n_items = nullptr;            // device copy of the call's item count
    int64_t *d_n_pairs = nullptr;            // pairs of the last call
    int64_t *d_status = nullptr;             // [0] status bits, [1] max pairs needed

    // profiling hooks
    cudaEvent_t prof_ev[4] = {nullptr, nullptr, nullptr, nullptr};
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
                          float *grad, int accumulate, cudaStream_t st);
}  // namespace vbm
