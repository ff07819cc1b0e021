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
void *g_ptr[kMaxDevices];   // device address of the scratch array, per device

// The array's name is only a host-side handle in host code: its device
// address has to be asked for once per device, with that device current.
hd_status scratch_address(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return HD_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return HD_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_hd_static_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return HD_ERR_CUDA;
        }
        g_ptr[dev] = p;
    }
    *out = g_ptr[dev];
    return HD_OK;
}

}  // namespace

extern "C" hd_status hybrid_denoise_static(const hd_image *img, hd_stream_t stream)
{
    if (!img) return HD_ERR_ARG;
    if (img->H < 1 || img->W < 1) return HD_ERR_ARG;
    size_t need = 0;
    // the smallest workspace is enough; the (mu, s2) plane is used when it fits too
    hd_status st = hybrid_min_workspace_size(img->H, img->W, img->dtype, &img->p, &need);
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
