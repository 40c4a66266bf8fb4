// gsrf_static.cu -- gsrf_render_static: the one-call render with its workspace in a
// fixed device array compiled into the library, for callers that cannot allocate
// device memory.
//
// Who cannot allocate: hosts that forbid device allocation once they are running
// (real-time or embedded loops that allocate everything at start-up), plugins inside an
// application whose own allocator owns all device memory, and code held to a fixed
// device-memory budget.  Such callers still pass their own inputs and outputs; only
// the intermediate workspace comes from this array.
//
// The array (GSRF_STATIC_SCRATCH_BYTES) is allocated by the CUDA driver when the
// library's module is loaded on a device and stays allocated on every device that
// loads the library until the process exits.  Every call made outside a stream capture
// looks up the array's device address (cudaGetSymbolAddress); make the first call on a
// device before any stream capture.  All calls share it and it keeps the
// previous call's contents; the render pipeline initialises everything it reads (its
// status word, list ranges and receiver bases) at the start of each call, so nothing
// has to be cleared by hand.  Two calls whose work overlaps on the GPU (different
// streams or host threads) race on the array and corrupt each other's results.
#include <mutex>

#include "gsrf_internal.cuh"

namespace gsrf {

static __device__ __align__(256) unsigned char g_static_scratch[GSRF_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
static void* g_scratch_ptr[kMaxDevices];
static std::mutex g_scratch_mu;

// Device address of the array on the current device.  The host-side name of the array
// is only a stand-in; its device address must come from cudaGetSymbolAddress with that
// device current.  Outside a stream capture the address is looked up again on every call
// (cheap once the module is loaded), so a cudaDeviceReset, after which the module is
// loaded afresh and the array may sit elsewhere, never leaves a stale address behind.
// During a capture the lookup is not made (it is not a stream operation); the address
// cached by the last call made outside a capture on this device is used, and a device
// that has had no such call is refused.
static cudaError_t scratch_on_current_device(cudaStream_t stream, void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if ((e = cudaStreamIsCapturing(stream, &cap)) != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        if (((uintptr_t)p & 255) != 0) return cudaErrorMisalignedAddress;
        g_scratch_ptr[dev] = p;
    } else if (!g_scratch_ptr[dev]) {
        return cudaErrorStreamCaptureUnsupported;
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace gsrf

using namespace gsrf;

extern "C" gsrf_status gsrf_render_static(const gsrf_plan* plan, const gsrf_gaussians* g, const float* rx_pos,
                                          const float* tx_pos, float* out_rays, gsrf_run_status* status,
                                          void* stream) {
    size_t need = 0;
    gsrf_status s = gsrf_workspace_size(plan, &need);
    if (s != GSRF_OK) return s;
    if (need > (size_t)GSRF_STATIC_SCRATCH_BYTES) return GSRF_ERR_TOO_LARGE;
    void* ws = nullptr;
    if (scratch_on_current_device((cudaStream_t)stream, &ws) != cudaSuccess) return GSRF_ERR_CUDA;
    s = gsrf_render(plan, g, rx_pos, tx_pos, ws, (size_t)GSRF_STATIC_SCRATCH_BYTES, out_rays, nullptr, stream);
    if (s != GSRF_OK || !status) return s;
    return gsrf_read_status(ws, (size_t)GSRF_STATIC_SCRATCH_BYTES, status, stream);
}
