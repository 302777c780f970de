// fd4_fed_cycle_noalloc: the FED cycle for callers that cannot allocate device
// memory.  Some host applications own every byte of device memory and hand a
// library only the buffers it works on (plugins inside a larger imaging
// pipeline with a fixed memory budget); others must not call cudaMalloc once
// they are running, because it can synchronise the device and break a
// latency budget, or because their code runs under a no-allocation policy
// after start-up.  Those callers cannot provide the workspace fd4_fed_cycle
// asks for, so this entry point uses a scratch buffer that lives in the
// library itself: a file-scope __device__ array that every GPU which loads
// the library holds until the process exits.
#include <cuda.h>

#include <mutex>

#include "fd4_internal.h"

namespace {

// Header slot (unused here, kept so the array has the workspace layout the
// FED launcher expects) followed by one float plane of up to
// FD4_NOALLOC_MAX_PIXELS pixels (h * pitch).
constexpr size_t kScratchBytes = fd4::kHeaderBytes + (size_t)FD4_NOALLOC_MAX_PIXELS * sizeof(float);
static __device__ __align__(256) unsigned char g_fed_scratch[kScratchBytes];

// In host code the array's name is only a host-side stand-in, so its device
// address is looked up with cudaGetSymbolAddress, with the device current,
// and cached per device together with the identity of the context it belongs
// to.  A device reset (cudaDeviceReset) ends that context and the array moves
// with the module into the next one: a call that finds another context looks
// the address up again instead of passing a stale one to the kernel.
struct ScratchAddr {
    void *addr;
    unsigned long long ctx_id;
};
constexpr int kMaxDevices = 64;
std::mutex g_mutex;
ScratchAddr g_scratch[kMaxDevices] = {};

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

template <class Fn>
Fn driver_fn(const char *name)
{
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
        return nullptr;
    return reinterpret_cast<Fn>(p);
}

// Identity of the calling thread's current context (false if none is current).
bool current_ctx_id(unsigned long long *id)
{
    static const CtxGetCurrentFn get_current = driver_fn<CtxGetCurrentFn>("cuCtxGetCurrent");
    static const CtxGetIdFn get_id = driver_fn<CtxGetIdFn>("cuCtxGetId");
    CUcontext ctx = nullptr;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return get_id(ctx, id) == CUDA_SUCCESS;
}

// Device address of g_fed_scratch on the current device.
int scratch_for_current_device(char **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FD4_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return FD4_ERR_BAD_ARG;
    unsigned long long id = 0;
    const bool have_id = current_ctx_id(&id);
    std::lock_guard<std::mutex> lock(g_mutex);
    ScratchAddr &c = g_scratch[dev];
    if (c.addr && have_id && c.ctx_id == id) {
        *out = (char *)c.addr;
        return FD4_OK;
    }
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_fed_scratch) != cudaSuccess || !p) return FD4_ERR_CUDA;
    // the look-up made the device's context current on this thread
    if (current_ctx_id(&id)) {
        c.addr = p;
        c.ctx_id = id;
    } else {
        c.addr = nullptr;  // no context identity: look the address up on every call
    }
    *out = (char *)p;
    return FD4_OK;
}

}  // namespace

extern "C" int fd4_fed_cycle_noalloc(float *d_u, int w, int h, int pitch, const float *d_tensor,
                                     const double *h_tau, int n, int boundary, fd4_stream_t stream)
{
    int rc;
    if ((rc = fd4::check_image(d_u, w, h, pitch)) != FD4_OK) return rc;
    if (!d_tensor || !h_tau || n < 1 || n > FD4_MAX_FED_STEPS) return FD4_ERR_BAD_ARG;
    if ((uintptr_t)d_tensor & 15u) return FD4_ERR_ALIGN;
    if (boundary != FD4_BC_NATURAL && boundary != FD4_BC_PERIODIC) return FD4_ERR_BAD_ARG;
    for (int i = 0; i < n; ++i)
        if (!(h_tau[i] > 0.0) || !(h_tau[i] < 1e6)) return FD4_ERR_BAD_ARG;
    if ((size_t)h * (size_t)pitch > (size_t)FD4_NOALLOC_MAX_PIXELS) return FD4_ERR_WS_TOO_SMALL;
    char *ws = nullptr;
    if ((rc = scratch_for_current_device(&ws)) != FD4_OK) return rc;
    // The scratch plane is written in full before it is read, so nothing in it
    // needs clearing between calls.
    if (fd4::launch_fed_cycle(d_u, w, h, pitch, d_tensor, h_tau, n, boundary, fd4::kDefaultSched, ws,
                              (cudaStream_t)stream))
        return FD4_ERR_CUDA;
    return FD4_OK;
}
