// vbm_loss_static: the image loss of vbm_loss with its scratch in a fixed
// device array of this library instead of a caller-provided workspace.
//
// Some callers cannot allocate device memory when they need the loss: code
// that runs while a CUDA graph is being captured (allocation is not allowed
// there), render or training loops whose memory budget is fixed when they
// start, and host programs that own only the image buffers they pass in.
// This entry point allocates nothing.  Its scratch is the file-scope array
// below (kStaticLossBytes = 32 MiB), which every GPU that loads the library
// holds until the process exits.
//
// The array's name is a host-side stand-in in host code, not a device
// address: the host looks up the device address once per device with
// cudaGetSymbolAddress and passes that pointer to the kernels.  The first
// call on a device does this and also uploads the SSIM window to that
// device's constant memory (a synchronous copy), so that first call should
// come before any stream capture.  All calls share the array and it keeps
// the last call's contents; every scratch word the loss kernels read is
// written earlier in the same call, so nothing has to be cleared.  Calls
// whose kernels overlap on the GPU (different streams, or different host
// threads) race on the array.
#include <mutex>

#include "vbm_internal.h"

namespace vbm {

size_t loss_workspace_bytes(int n_images, int H, int W);
vbm_status loss_fwd_bwd(const float *img, const float *target, int n_images, int H, int W, float lambda,
                        double scale, double *loss, int accumulate, float *dimg, void *ws, cudaStream_t st);

namespace {

constexpr size_t kStaticLossBytes = size_t(32) << 20;

static __device__ __align__(256) unsigned char g_static_loss_scratch[kStaticLossBytes];

constexpr int kMaxDevices = 64;
std::mutex g_symbol_mutex;
void *g_symbol_addr[kMaxDevices] = {};

vbm_status static_scratch(void **out)
{
    int dev = 0;
    VBM_CUDA(cudaGetDevice(&dev));
    VBM_ARG(dev >= 0 && dev < kMaxDevices, "device index out of range");
    std::lock_guard<std::mutex> lock(g_symbol_mutex);
    if (!g_symbol_addr[dev]) {
        void *ptr = nullptr;
        VBM_CUDA(cudaGetSymbolAddress(&ptr, g_static_loss_scratch));
        g_symbol_addr[dev] = ptr;
    }
    *out = g_symbol_addr[dev];
    return VBM_OK;
}

}  // namespace
}  // namespace vbm

extern "C" {

vbm_status vbm_loss_static(const float *img, const float *target, int n_images, int height, int width,
                           float lambda, double scale, double *loss, int32_t accumulate, float *dimg, void *stream)
{
    VBM_ARG(img && target && loss && dimg, "null argument");
    VBM_ARG(n_images > 0 && height > 0 && width > 0, "invalid image size");
    const size_t need = vbm::loss_workspace_bytes(n_images, height, width);
    if (need > vbm::kStaticLossBytes) {
        vbm::set_error("vbm_loss_static: " + std::to_string(n_images) + " images of " + std::to_string(width) + "x" +
                       std::to_string(height) + " need " + std::to_string(need) + " bytes of scratch, more than the " +
                       std::to_string(vbm::kStaticLossBytes) + "-byte static array; call it per image (accumulate) "
                       "or use vbm_loss with a workspace");
        return VBM_ERR_CAPACITY;
    }
    void *ws = nullptr;
    vbm_status s = vbm::static_scratch(&ws);
    if (s != VBM_OK) return s;
    return vbm::loss_fwd_bwd(img, target, n_images, height, width, lambda, scale, loss, accumulate, dimg, ws,
                             (cudaStream_t)stream);
}

}  // extern "C"
