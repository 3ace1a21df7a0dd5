// L1 + D-SSIM loss with scratch that the library owns, for callers that must
// not allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocating routine) where they
// compute the loss: a plug-in living inside another framework's memory pool,
// a process that reserves all device memory up front and must not grow it,
// or a latency-critical loop that must never enter the driver's allocator.
// mvgs_dssim_loss needs a caller-sized workspace; this variant instead uses a
// fixed file-scope device array, so the caller passes only the images, the
// targets and the outputs.
//
// The array is static device storage: every GPU that loads the library holds
// kScratchBytes of it until the process exits.  Its device address is looked
// up on every call made outside stream capture and cached per device; a call
// under capture uses the cached address, so a device's first call must come
// before any capture (a first call under capture returns MVGS_ECUDA without
// launching).  All calls share the array and it keeps the previous call's
// contents; the loss kernels write every scratch value before reading it, so
// nothing needs clearing, but calls that overlap on the GPU (different
// streams, no ordering between them) race on the array.
#include <mutex>
#include <unordered_map>

#include "../../include/mvgs.h"
#include "kernels.h"

namespace {

// 80 MiB: one 1920x1080 view (about 75 MB of scratch), or several smaller
// views totalling about 2.2 million pixels.
constexpr size_t kScratchBytes = 80ull << 20;

static __device__ __align__(256) unsigned char g_dssim_scratch[kScratchBytes];

std::mutex g_mu;
std::unordered_map<int, void*> g_device_ptr;

// Device address of the scratch array on the current device (nullptr and a
// CUDA error when the lookup fails).  Looked up again on every call that is
// not under stream capture (the address follows the device's current
// context, e.g. after cudaDeviceReset); a call under capture takes the
// address cached by the device's last call outside capture.
void* scratch_ptr(cudaStream_t stream, cudaError_t& err) {
    int dev = 0;
    err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return nullptr;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    err = cudaStreamIsCapturing(stream, &cap);
    if (err != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    if (cap != cudaStreamCaptureStatusNone) {
        auto it = g_device_ptr.find(dev);
        if (it == g_device_ptr.end()) err = cudaErrorStreamCaptureUnsupported;
        return it == g_device_ptr.end() ? nullptr : it->second;
    }
    void* p = nullptr;
    err = cudaGetSymbolAddress(&p, g_dssim_scratch);
    if (err != cudaSuccess || p == nullptr) return nullptr;
    g_device_ptr[dev] = p;
    return p;
}

}  // namespace

extern "C" mvgs_status mvgs_dssim_loss_noalloc(const float* img, const float* target, const int32_t* hw, int32_t V,
                                               float lambda, float* loss_per_view, float* dL_dimg,
                                               mvgs_stream stream) {
    using namespace mvgs;
    auto record_error = [](int st, const char* msg) { return (mvgs_status)mvgs::record_error(st, msg); };
    if (!img || !target || !hw || !loss_per_view) return record_error(MVGS_EINVAL, "NULL argument");
    if (V < 1) return record_error(MVGS_EINVAL, "need at least one view");
    for (int v = 0; v < V; v++)
        if (hw[2 * v] < 1 || hw[2 * v + 1] < 1) return record_error(MVGS_EINVAL, "empty image");
    if (!(lambda >= 0.f && lambda <= 1.f)) return record_error(MVGS_EINVAL, "lambda must be in [0, 1]");
    const size_t need = dssim_temp_bytes(hw, V);
    if (need > kScratchBytes)
        return record_error(MVGS_ENOSPACE,
                            "these views need more scratch than the library's static buffer holds "
                            "(80 MiB, about 2.2 million pixels per call); use mvgs_dssim_loss with a workspace");
    cudaError_t err = cudaSuccess;
    const cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    void* scratch = scratch_ptr(s, err);
    if (!scratch) return record_error(MVGS_ECUDA, cudaGetErrorString(err));
    {
        StageTimer t(MVGS_STAGE_DSSIM, s);
        launch_dssim(img, target, hw, V, lambda, loss_per_view, dL_dimg, scratch, s);
    }
    err = cudaGetLastError();
    if (err != cudaSuccess) return record_error(MVGS_ECUDA, cudaGetErrorString(err));
    return MVGS_OK;
}
