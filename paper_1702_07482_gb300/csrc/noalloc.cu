// tnrd_forward_noalloc: the fused forward cascade with its inter-stage image
// in a scratch array compiled into the library, for callers that cannot
// allocate device memory (see include/tnrd.h).
#include "tnrd.h"
#include "launch.h"

#include <cuda_runtime.h>
#include <cstdio>
#include <mutex>

namespace {

// The scratch: one array per GPU that loads the library, alive until exit.
// In host code this name is only a host-side stand-in, not a device address;
// the device address is looked up once per device with cudaGetSymbolAddress.
__device__ __align__(256) float g_noalloc_scratch[TNRD_NOALLOC_MAX_FLOATS];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
// Per device: the array's device address and the id of the context it was
// looked up in.  A device reset (cudaDeviceReset) ends that context and may
// load the module, and with it the array, at another address; a call in a new
// context therefore looks the address up again instead of using a stale one.
struct ScratchSlot {
    unsigned long long ctx;
    float* ptr;
};
ScratchSlot g_scratch[kMaxDevices] = {};

}  // namespace

extern "C" tnrd_status tnrd_forward_noalloc(const tnrd_params* params, int N, int H, int W,
                                            int pitch, const float* f, float* u,
                                            cudaStream_t stream)
{
    // The size check comes before any CUDA call, so nothing is launched for a
    // batch that does not fit; tnrd_forward validates everything else.
    if (N > 0 && H > 0 && pitch > 0 &&
        (unsigned long long)N * (unsigned long long)H * (unsigned long long)pitch >
            (unsigned long long)TNRD_NOALLOC_MAX_FLOATS) {
        char msg[256];
        snprintf(msg, sizeof msg,
                 "tnrd_forward_noalloc: N*H*pitch = %llu floats exceeds the built-in scratch "
                 "of %u floats (TNRD_NOALLOC_MAX_FLOATS); use tnrd_forward with a workspace",
                 (unsigned long long)N * H * pitch, (unsigned)TNRD_NOALLOC_MAX_FLOATS);
        return tnrd::set_error(TNRD_ERR_INVALID_ARG, msg);
    }
    if (N <= 0 || H <= 0 || pitch <= 0)   // no-op or invalid: tnrd_forward says which
        return tnrd_forward(params, N, H, W, pitch, f, u, 0, TNRD_ALGO_FUSED, nullptr, 0, stream);

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return tnrd::set_error(TNRD_ERR_CUDA, "tnrd_forward_noalloc: cudaGetDevice failed");
    }
    if (dev < 0 || dev >= kMaxDevices)
        return tnrd::set_error(TNRD_ERR_UNSUPPORTED, "tnrd_forward_noalloc: device index too large");
    float* scratch;
    {
        // Set-up, once per device (and again in a new context), with that
        // device current.
        std::lock_guard<std::mutex> lock(g_mu);
        ScratchSlot& slot = g_scratch[dev];
        const unsigned long long ctx = tnrd::current_context_id();
        if (!slot.ptr || ctx == 0 || ctx != slot.ctx) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                (void)cudaGetLastError();   // leave no stale error for the caller's next check
                slot.ptr = nullptr;
                char msg[256];
                snprintf(msg, sizeof msg,
                         "tnrd_forward_noalloc: cudaGetSymbolAddress of the scratch failed: %s (%s)",
                         cudaGetErrorName(e), cudaGetErrorString(e));
                return tnrd::set_error(TNRD_ERR_CUDA, msg);
            }
            slot.ptr = static_cast<float*>(p);
            slot.ctx = tnrd::current_context_id();   // the lookup may have made it current
        }
        scratch = slot.ptr;
    }
    // The scratch holds the image between stages; it is always written before
    // it is read, so it needs no clearing.
    return tnrd_forward(params, N, H, W, pitch, f, u, 0, TNRD_ALGO_FUSED, scratch,
                        sizeof(float) * (size_t)TNRD_NOALLOC_MAX_FLOATS, stream);
}
