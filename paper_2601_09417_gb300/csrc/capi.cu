// extern "C" entry points of libvbm: argument checks, plan ownership and
// dispatch to the kernels of the other translation units.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cstring>
#include <string>

#include "vbm_internal.h"

namespace vbm {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

vbm_status cuda_fail(cudaError_t e, const char *what)
{
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? VBM_ERR_NOMEM : VBM_ERR_CUDA;
}

static std::atomic<int64_t> g_launches{0};

void note_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void record_event(cudaEvent_t ev, cudaStream_t st)
{
    if (!ev) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    if (cs == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal);
    else cudaEventRecord(ev, st);
}

int num_sms()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

size_t loss_workspace_bytes(int n_images, int H, int W);
vbm_status loss_fwd_bwd(const float *img, const float *target, int n_images, int H, int W, float lambda,
                        double scale, double *loss, int accumulate, float *dimg, void *ws, cudaStream_t st);
vbm_status adam_step(float *P, const float *G, float *M, float *V, int64_t n, int64_t stride, int32_t *step,
                     const float lrs[5], float beta1, float beta2, float eps, uint32_t *nonfinite, cudaStream_t st);
vbm_status render_dvr(const float *F, const int dims[3], const vbm_tf *tf, const vbm_camera *cams, int n_views,
                      int W, int H, float step, float *out, cudaStream_t st);

template <typename T>
static vbm_status plan_alloc(vbm_plan *p, T **ptr, size_t count)
{
    void *q = nullptr;
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) return cuda_fail(e, "plan allocation");
    p->allocations.push_back(q);
    *ptr = (T *)q;
    return VBM_OK;
}

static void plan_free(vbm_plan *p)
{
    for (void *q : p->allocations) cudaFree(q);
    p->allocations.clear();
}

}  // namespace vbm

using namespace vbm;

extern "C" {

const char *vbm_last_error(void) { return g_last_error.c_str(); }

int vbm_version(void) { return 101; }

int64_t vbm_kernel_launches(void) { return g_launches.load(); }

vbm_status vbm_plan_set_profile(vbm_plan *p, int32_t n_events, void *const *events, int32_t *d_n_eval,
                                int32_t *d_n_contrib)
{
    VBM_ARG(p, "null plan");
    VBM_ARG(n_events == 0 || n_events == 4 || n_events == kProfileEvents, "n_events must be 0, 4 or 7");
    VBM_ARG(n_events == 0 || events, "null events");
    for (int i = 0; i < kProfileEvents; i++) p->prof_ev[i] = i < n_events ? (cudaEvent_t)events[i] : nullptr;
    p->prof_n_eval = d_n_eval;
    p->prof_n_contrib = d_n_contrib;
    return VBM_OK;
}

vbm_status vbm_plan_create(const vbm_plan_desc *d, vbm_plan **out)
{
    VBM_ARG(d && out, "null argument");
    VBM_ARG(d->n_scenes >= 1 && d->n_views >= 1, "need at least one scene and one view");
    VBM_ARG(d->scene_offset != nullptr, "scene_offset is required");
    VBM_ARG(d->n_scenes == 1 || d->view_scene != nullptr, "view_scene is required with several scenes");
    VBM_ARG(d->width > 0 && d->height > 0, "image size must be positive");
    const int tp = d->tile_w * d->tile_h;
    VBM_ARG((d->tile_w == 8 || d->tile_w == 16) && d->tile_h > 0 && d->tile_h % 4 == 0 &&
                (tp == 32 || tp == 64 || tp == 128 || tp == 256),
            "tile_w must be 8 or 16, tile_h a multiple of 4 and tile_w * tile_h 32, 64, 128 or 256");
    VBM_ARG(d->group_lanes == 0 || d->group_lanes == 4 || d->group_lanes == 8 || d->group_lanes == 16 ||
                d->group_lanes == 32,
            "group_lanes must be 0, 4, 8, 16 or 32");
    VBM_ARG(d->pair_capacity > 0 && d->pair_capacity < ((int64_t)1 << 31), "pair_capacity out of range");
    VBM_ARG(d->pixels_per_thread == 0 || d->pixels_per_thread == 1 || d->pixels_per_thread == 2 ||
                d->pixels_per_thread == 4,
            "pixels_per_thread must be 0, 1, 2 or 4");
    VBM_ARG(d->bwd_group_lanes == 0 || d->bwd_group_lanes == 4 || d->bwd_group_lanes == 8 ||
                d->bwd_group_lanes == 16 || d->bwd_group_lanes == 32,
            "bwd_group_lanes must be 0, 4, 8, 16 or 32");
    VBM_ARG(d->bwd_pixels_per_thread == 0 || d->bwd_pixels_per_thread == 1 || d->bwd_pixels_per_thread == 2 ||
                d->bwd_pixels_per_thread == 4,
            "bwd_pixels_per_thread must be 0, 1, 2 or 4");
    VBM_ARG(d->segment_len == -1 || (d->segment_len >= 0 && d->segment_len <= 65536 && d->segment_len % 32 == 0),
            "segment_len must be -1, 0 or a positive multiple of 32 up to 65536");
    VBM_ARG((d->width + d->tile_w - 1) / d->tile_w <= kMaxTilesPerAxis &&
                (d->height + d->tile_h - 1) / d->tile_h <= kMaxTilesPerAxis,
            "at most 65535 tiles along each image axis");
    VBM_ARG(d->scene_offset[0] == 0, "scene_offset[0] must be 0");
    for (int s = 0; s < d->n_scenes; s++)
        VBM_ARG(d->scene_offset[s + 1] >= d->scene_offset[s], "scene_offset must be non-decreasing");
    if (d->view_scene)
        for (int v = 0; v < d->n_views; v++)
            VBM_ARG(d->view_scene[v] >= 0 && d->view_scene[v] < d->n_scenes, "view_scene out of range");
    vbm_plan *p = new vbm_plan();
    p->desc = *d;
    p->scene_offset.assign(d->scene_offset, d->scene_offset + d->n_scenes + 1);
    if (d->view_scene) p->view_scene.assign(d->view_scene, d->view_scene + d->n_views);
    else p->view_scene.assign(d->n_views, 0);
    p->desc.scene_offset = nullptr;
    p->desc.view_scene = nullptr;
    p->TX = (d->width + d->tile_w - 1) / d->tile_w;
    p->TY = (d->height + d->tile_h - 1) / d->tile_h;
    p->n_gauss = p->scene_offset[d->n_scenes];
    p->view_item_offset.assign(d->n_views + 1, 0);
    for (int v = 0; v < d->n_views; v++) {
        int s = p->view_scene[v];
        int64_t ns = p->scene_offset[s + 1] - p->scene_offset[s];
        p->view_item_offset[v + 1] = p->view_item_offset[v] + ns;
        p->max_scene = std::max(p->max_scene, ns);
    }
    p->items_cap = p->view_item_offset[d->n_views];
    if (p->items_cap >= ((int64_t)1 << 32) - 1) {
        delete p;
        set_error("too many (view, Gaussian) items for 32-bit item indices");
        return VBM_ERR_ARG;
    }
    // scene -> views (CSR)
    std::vector<int32_t> ptr(d->n_scenes + 1, 0), views;
    for (int v = 0; v < d->n_views; v++) ptr[p->view_scene[v] + 1]++;
    for (int s = 0; s < d->n_scenes; s++) ptr[s + 1] += ptr[s];
    views.resize(d->n_views);
    std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
    for (int v = 0; v < d->n_views; v++) views[fill[p->view_scene[v]]++] = v;

    const int64_t items = p->items_cap, pairs = d->pair_capacity;
    const int64_t tiles = (int64_t)d->n_views * p->TX * p->TY;
    const int64_t pixels = (int64_t)d->n_views * d->width * d->height;
    vbm_status s = VBM_OK;
#define ALLOC(ptr_, n_)                                   \
    if (s == VBM_OK) s = plan_alloc(p, &(ptr_), (size_t)(n_))
    ALLOC(p->d_scene_offset, d->n_scenes + 1);
    ALLOC(p->d_view_scene, d->n_views);
    ALLOC(p->d_view_item_offset, d->n_views + 1);
    ALLOC(p->d_scene_view_ptr, d->n_scenes + 1);
    ALLOC(p->d_scene_views, d->n_views);
    ALLOC(p->rec, items);
    ALLOC(p->place, items);
    ALLOC(p->g_splat, kGradStride * items);
    ALLOC(p->pair_key, pairs);
    ALLOC(p->pair_tile, pairs);
    ALLOC(p->pair_item, pairs);
    ALLOC(p->tile_count, tiles);
    ALLOC(p->ranges, tiles);
    ALLOC(p->tile_order, tiles);
    ALLOC(p->tile_queue, kTileQueueWords);
    if ((d->flags & VBM_PLAN_PERSISTENT) && d->segment_len >= 0) {
        p->seg_len = d->segment_len ? d->segment_len : kDefaultSegmentLen;
        const int64_t tile_px = (int64_t)d->tile_w * d->tile_h;
        // boundary slots for about kCheckpointPairsPerItem pairs per item (the
        // workloads list about two per item before fine-tuning shrinks the
        // splats, fewer after), one final-state slot per tile in recompute
        // plans; never more than the pair capacity can use or kCheckpointBytes
        const bool rc = (d->flags & VBM_PLAN_RECOMPUTE) != 0;
        const int64_t want = (kCheckpointPairsPerItem * items + p->seg_len - 1) / p->seg_len + (rc ? tiles : 0);
        const int64_t usable = (pairs + p->seg_len - 1) / p->seg_len * (rc ? 2 : 1);
        p->ckpt_cap = std::max<int64_t>(1, std::min({want, usable,
                                                     kCheckpointBytes / (tile_px * (int64_t)sizeof(float4))}));
        ALLOC(p->ckpt, p->ckpt_cap * tile_px);
        ALLOC(p->ckpt_base, tiles);
        ALLOC(p->seg_units, 2 * p->ckpt_cap);
    }
    if (d->flags & VBM_PLAN_RADIX_SORT) {
        p->radix_blocks = radix_blocks();
        p->scan_blocks = scan_blocks();
        ALLOC(p->touched, items);
        for (int k = 0; k < 2; k++) {
            ALLOC(p->item_key[k], items);
            ALLOC(p->item_val[k], items);
        }
        ALLOC(p->item_offset, items + 1);
        ALLOC(p->d_n_items, 1);
        ALLOC(p->radix_hist, radix_hist_words(p->radix_blocks));
        ALLOC(p->radix_total, 256);
        ALLOC(p->scan_sums, p->scan_blocks + 1);
    }
    if (!(d->flags & VBM_PLAN_RECOMPUTE)) {
        ALLOC(p->T_final, pixels);
        ALLOC(p->n_contrib, pixels);
    }
    p->bin_scratch.chunks = bin_chunks(tiles);
    ALLOC(p->bin_scratch.chunk_sums, p->bin_scratch.chunks);
    ALLOC(p->bin_scratch.long_tiles, 2 * tiles);
    ALLOC(p->bin_scratch.long_count, 3);
    ALLOC(p->d_n_pairs, 1);
    ALLOC(p->d_status, 2);
#undef ALLOC
    if (s != VBM_OK) {
        plan_free(p);
        delete p;
        return s;
    }
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaMemcpy(p->d_scene_offset, p->scene_offset.data(), sizeof(int64_t) * (d->n_scenes + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_view_scene, p->view_scene.data(), sizeof(int32_t) * d->n_views, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_view_item_offset, p->view_item_offset.data(), sizeof(int64_t) * (d->n_views + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_scene_view_ptr, ptr.data(), sizeof(int32_t) * (d->n_scenes + 1), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_scene_views, views.data(), sizeof(int32_t) * d->n_views, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(p->d_status, 0, 2 * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMemset(p->d_n_pairs, 0, sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMemset(p->tile_count, 0, sizeof(uint32_t) * std::max<int64_t>(tiles, 1));
    if (e == cudaSuccess) e = binning_setup();
    if (e != cudaSuccess) {
        plan_free(p);
        delete p;
        return cuda_fail(e, "plan initialisation");
    }
    *out = p;
    return VBM_OK;
}

vbm_status vbm_plan_destroy(vbm_plan *p)
{
    if (!p) return VBM_OK;
    cudaDeviceSynchronize();
    plan_free(p);
    delete p;
    return VBM_OK;
}

vbm_status vbm_plan_check(vbm_plan *p, void *stream, int64_t *pairs_needed)
{
    VBM_ARG(p, "null plan");
    cudaStream_t st = (cudaStream_t)stream;
    int64_t h[2] = {0, 0};
    VBM_CUDA(cudaMemcpyAsync(h, p->d_status, sizeof(h), cudaMemcpyDeviceToHost, st));
    VBM_CUDA(cudaStreamSynchronize(st));
    VBM_CUDA(cudaMemsetAsync(p->d_status, 0, sizeof(h), st));
    VBM_CUDA(cudaStreamSynchronize(st));
    if (pairs_needed) *pairs_needed = h[1];
    if (h[0] & kStatusCapacity) {
        set_error("pair capacity exceeded: " + std::to_string(h[1]) + " pairs needed, capacity " +
                  std::to_string(p->desc.pair_capacity));
        return VBM_ERR_CAPACITY;
    }
    return VBM_OK;
}

static vbm_status check_call(vbm_plan *p, const float *params, int64_t stride, const vbm_camera *cams, int vb,
                             int vc)
{
    VBM_ARG(p && cams, "null argument");
    VBM_ARG(params || p->n_gauss == 0, "null parameter array");
    VBM_ARG(vb >= 0 && vc >= 1 && vb + vc <= p->desc.n_views, "view range out of bounds");
    VBM_ARG(stride >= p->n_gauss, "stride smaller than the number of Gaussians");
    return VBM_OK;
}

vbm_status vbm_raster_fwd(vbm_plan *p, const float *params, int64_t stride, const vbm_camera *cams, int32_t vb,
                          int32_t vc, const float bg[3], float *img, float *alpha, void *stream)
{
    vbm_status s = check_call(p, params, stride, cams, vb, vc);
    if (s != VBM_OK) return s;
    VBM_ARG(bg && img, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    p->last_view_begin = vb;
    p->last_view_count = vc;
    p->last_items = p->view_item_offset[vb + vc] - p->view_item_offset[vb];
    p->g_splat_clear = p->bwd_seen;   // the projection zeroes the items' splat-gradient records
    p->bwd_queue_used = false;        // the binning zeroes the work-queue counters
    record_event(p->prof_ev[4], st);
    s = preprocess_fwd(p, params, stride, cams, vb, vc, st);
    record_event(p->prof_ev[5], st);
    if (s == VBM_OK) s = binning(p, vb, vc, st);
    if (s == VBM_OK) s = raster_fwd(p, vb, vc, bg, img, alpha, st);
    return s;
}

vbm_status vbm_raster_bwd(vbm_plan *p, const float *params, int64_t stride, const vbm_camera *cams, int32_t vb,
                          int32_t vc, const float bg[3], const float *dimg, const float *dalpha, float *grad,
                          int32_t accumulate, void *stream)
{
    vbm_status s = check_call(p, params, stride, cams, vb, vc);
    if (s != VBM_OK) return s;
    VBM_ARG(bg && dimg && grad, "null argument");
    VBM_ARG(vb == p->last_view_begin && vc == p->last_view_count,
            "backward views differ from the last forward call on this plan");
    cudaStream_t st = (cudaStream_t)stream;
    s = raster_bwd(p, params, stride, vb, vc, bg, dimg, dalpha, grad, st);
    if (s == VBM_OK) s = preprocess_bwd(p, params, stride, cams, vb, vc, grad, accumulate, st);
    record_event(p->prof_ev[6], st);
    return s;
}

vbm_status vbm_raster_bwd_adam(vbm_plan *p, float *params, int64_t stride, const vbm_camera *cams, int32_t vb,
                               int32_t vc, const float bg[3], const float *dimg, const float *dalpha, float *m, float *v,
                               int64_t n, int32_t *step, const float lrs[5], float beta1, float beta2, float eps,
                               uint32_t *nonfinite, void *stream)
{
    vbm_status s = check_call(p, params, stride, cams, vb, vc);
    if (s != VBM_OK) return s;
    VBM_ARG(bg && dimg && m && v && step && lrs, "null argument");
    VBM_ARG(n >= 0 && stride >= n, "invalid size");
    VBM_ARG(vb == p->last_view_begin && vc == p->last_view_count,
            "backward views differ from the last forward call on this plan");
    cudaStream_t st = (cudaStream_t)stream;
    AdamArgs a;
    a.P = params;
    a.M = m;
    a.V = v;
    a.step = step;
    a.n = n;
    for (int k = 0; k < 5; k++) a.lr[k] = lrs[k];
    a.beta1 = beta1;
    a.beta2 = beta2;
    a.eps = eps;
    a.nonfinite = nonfinite;
    s = raster_bwd(p, params, stride, vb, vc, bg, dimg, dalpha, nullptr, st);
    if (s == VBM_OK) s = adam_step_inc(step, st);
    if (s == VBM_OK) s = preprocess_bwd(p, params, stride, cams, vb, vc, nullptr, 0, st, &a);
    record_event(p->prof_ev[6], st);
    return s;
}

vbm_status vbm_plan_get_buffers(vbm_plan *p, vbm_plan_buffers *o)
{
    VBM_ARG(p && o, "null argument");
    std::memset(o, 0, sizeof(*o));
    o->n_items = p->last_items;
    o->rec = (const float *)p->rec;
    o->place = (const uint32_t *)p->place;
    o->pair_tile = p->pair_tile;
    o->pair_item = p->pair_item;
    o->ranges = (const int32_t *)p->ranges;
    o->n_pairs = p->d_n_pairs;
    o->T_final = p->T_final;
    o->n_contrib = p->n_contrib;
    o->g_splat = p->g_splat;
    o->seg_count = p->seg_len ? p->tile_queue + kQSegUnits : nullptr;
    o->checkpoint_slots = p->seg_len ? p->ckpt_cap : 0;
    return VBM_OK;
}

vbm_status vbm_loss_workspace_size(int n_images, int height, int width, size_t *bytes)
{
    VBM_ARG(bytes && n_images > 0 && height > 0 && width > 0, "invalid argument");
    *bytes = loss_workspace_bytes(n_images, height, width);
    return VBM_OK;
}

vbm_status vbm_loss(const float *img, const float *target, int n_images, int height, int width, float lambda,
                    double scale, double *loss, int32_t accumulate, float *dimg, void *ws, size_t ws_bytes,
                    void *stream)
{
    VBM_ARG(img && target && loss && dimg && ws, "null argument");
    VBM_ARG(n_images > 0 && height > 0 && width > 0, "invalid image size");
    VBM_ARG(ws_bytes >= loss_workspace_bytes(n_images, height, width), "loss workspace too small");
    return loss_fwd_bwd(img, target, n_images, height, width, lambda, scale, loss, accumulate, dimg, ws,
                        (cudaStream_t)stream);
}

vbm_status vbm_adam(float *params, const float *grad, float *m, float *v, int64_t n, int64_t stride,
                    int32_t *step, const float lrs[5], float beta1, float beta2, float eps, uint32_t *nonfinite,
                    void *stream)
{
    VBM_ARG(params && grad && m && v && step && lrs, "null argument");
    VBM_ARG(n >= 0 && stride >= n, "invalid size");
    return adam_step(params, grad, m, v, n, stride, step, lrs, beta1, beta2, eps, nonfinite, (cudaStream_t)stream);
}

vbm_status vbm_render_dvr(const float *volume, const int dims[3], const vbm_tf *tf, const vbm_camera *cams,
                          int n_views, int width, int height, float step, float *rgba, void *stream)
{
    VBM_ARG(volume && dims && tf && cams && rgba, "null argument");
    VBM_ARG(dims[0] > 0 && dims[1] > 0 && dims[2] > 0, "invalid volume size");
    VBM_ARG(n_views > 0 && width > 0 && height > 0, "invalid image size");
    VBM_ARG(step > 0.f, "step must be positive");
    VBM_ARG(tf->n_knots >= 2 && tf->n_knots <= 16, "n_knots must be in [2, 16]");
    for (int i = 1; i < tf->n_knots; i++) VBM_ARG(tf->x[i] > tf->x[i - 1], "TF knots must be ascending");
    return render_dvr(volume, dims, tf, cams, n_views, width, height, step, rgba, (cudaStream_t)stream);
}

}  // extern "C"
