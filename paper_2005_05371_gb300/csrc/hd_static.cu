// hd_static.cu -- hybrid_denoise_static: the hybrid denoise without any
// device allocation by the caller or by the library.
//
// Some callers cannot allocate device memory: code that runs where
// cudaMalloc is not allowed or would block (inside a real-time frame loop
// with a fixed memory budget, in a plug-in host that owns the CUDA
// allocator, or in a driver-side callback).  For them the scratch this
// path needs (the median-filtered plane kept between the two phases, the
// work-queue counters and, when it fits, the plane of binary32 local
// statistics) lives in one fixed array in device memory, declared
// below.  Every GPU that loads this library holds that array until the
// process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "hd_internal.h"
#include "hybrid_denoise.h"

namespace {

// Scratch shared by every call of hybrid_denoise_static on a device.
static __device__ __align__(256) unsigned char g_hd_static_scratch[HD_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct Cached {
    void *ptr;                   // device address of the scratch array
    unsigned long long ctx_id;   // context it was looked up in (0: unknown)
};
Cached g_cache[kMaxDevices];

// The identity of the calling thread's current context (CUDA driver
// cuCtxGetCurrent / cuCtxGetId, reached through the runtime's entry-point
// query so the library needs no link against the driver library).  A
// context that is destroyed and created again (cudaDeviceReset, then the
// next runtime call) gets a new identity, and the array may then sit at
// another address.  Returns false when the identity is not available.
typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);

bool current_context_id(unsigned long long *id)
{
    static CtxGetCurrentFn get_cur = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_cur = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f);
        cudaGetLastError();
    });
    if (!get_cur || !get_id) return false;
    void *ctx = nullptr;
    if (get_cur(&ctx) != 0 || !ctx) return false;
    return get_id(ctx, id) == 0 && *id != 0;
}

// In host code the array's name is only a host-side handle: its device
// address has to be asked for with the device current.  The address is
// looked up on the first call on each device and again whenever the
// current context is not the one it was looked up in.
hd_status scratch_address(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HD_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return HD_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    unsigned long long id = 0;
    const bool have_id = current_context_id(&id);
    Cached &c = g_cache[dev];
    if (!c.ptr || !have_id || c.ctx_id != id) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_hd_static_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return HD_ERR_CUDA;
        }
        // the lookup itself creates the context when none was current yet
        unsigned long long id2 = 0;
        c.ptr = p;
        c.ctx_id = current_context_id(&id2) ? id2 : 0;
    }
    *out = c.ptr;
    return HD_OK;
}

}  // namespace

extern "C" hd_status hybrid_denoise_static(const hd_image *img, hd_stream_t stream)
{
    // the same argument checks, in the same order, as hybrid_denoise; the
    // size limit of the fixed array comes after them
    hd_status st = (hd_status)hd::check_hybrid_image(img);
    if (st != HD_OK) return st;
    size_t need = 0;
    // the smallest workspace is enough; the (mu, s2) plane is used when it fits too
    st = hybrid_min_workspace_size(img->H, img->W, img->dtype, &img->p, &need);
    if (st != HD_OK) return st;
    if (need > HD_STATIC_SCRATCH_BYTES) return HD_ERR_OVERFLOW;
    void *scratch = nullptr;
    st = scratch_address(&scratch);
    if (st != HD_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    // the queue counters must start at zero; the previous call's median plane
    // may stay (it is overwritten before it is read)
    if (need > 0 && cudaMemsetAsync(scratch, 0, hd::hybrid_control_bytes(), s) != cudaSuccess)
        return HD_ERR_CUDA;
    return (hd_status)hd::hybrid_on_workspace(img, need > 0 ? scratch : nullptr, need > 0 ? HD_STATIC_SCRATCH_BYTES : 0,
                                              stream);
}
