// hd_refnoise.cu -- noise variance against a clean reference image.
//
// Algorithm 1, step 4d hands the original image to the Wiener stage.  The
// library reads that as the source of the noise variance: for the Wiener
// input f and the reference r,
//   nu2 = fl64( fl64(S) / N ),  S = sum over pixels of (f - r)^2  (exact integer),
// which the caller then passes as noise_var (the hybrid is then one fused
// pass with no image-wide dependency).
//
// One launch: CTAs stride over rows, each accumulates its part of S in 64-bit
// integers and adds it to the workspace with one atomic; the last CTA to
// finish (a counter, no waiting) forms nu2, writes it and zeroes the counters.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "hd_contrast.h"
#include "hd_internal.h"
#include "hybrid_denoise.h"

namespace hd {
namespace {

typedef unsigned int u32;
typedef unsigned long long u64;

constexpr int kRnThreads = 512;
constexpr int kRnWarps = kRnThreads / 32;

struct RnCtl {
    u64 sum;          // S so far
    u32 done;         // CTAs that added their part
    u32 pad[61];
};
static_assert(sizeof(RnCtl) == HD_REFNOISE_WORKSPACE_BYTES, "RnCtl layout");

struct RnParams {
    const uint8_t *f, *r;
    long long fp, rp;         // pitches, bytes
    u32 H, W;
    int elem;
    double *out;
    RnCtl *ctl;
};

template <int ES>
__device__ __forceinline__ u32 px(const uint8_t *row, u32 x)
{
    return ES == 1 ? (u32)row[x] : (u32) reinterpret_cast<const uint16_t *>(row)[x];
}

template <int ES>
__global__ void __launch_bounds__(kRnThreads) refnoise_kernel(RnParams p)
{
    __shared__ u64 s_part[kRnWarps];
    u64 acc = 0;
    for (u32 y = blockIdx.x; y < p.H; y += gridDim.x) {
        const uint8_t *fr = p.f + (long long)y * p.fp;
        const uint8_t *rr = p.r + (long long)y * p.rp;
        for (u32 x = threadIdx.x; x < p.W; x += kRnThreads) {
            const int d = (int)px<ES>(fr, x) - (int)px<ES>(rr, x);
            acc += (u64)((u32)(d * d));        // below 2^32
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31u) == 0) s_part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        u64 t = 0;
        for (int w = 0; w < kRnWarps; ++w) t += s_part[w];
        atomicAdd(&p.ctl->sum, t);
        __threadfence();
        const u32 old = atomicAdd(&p.ctl->done, 1u);
        if (old == gridDim.x - 1) {
            __threadfence();
            const u64 S = atomicAdd(&p.ctl->sum, 0ull);
            *p.out = __ddiv_rn(__ull2double_rn(S), (double)p.H * (double)p.W);
            p.ctl->sum = 0;
            p.ctl->done = 0;
            __threadfence();
        }
    }
}

}  // namespace
}  // namespace hd

using namespace hd;

extern "C" {

hd_status reference_noise_variance(const void *f, size_t f_pitch, const void *ref, size_t ref_pitch, int H, int W,
                                   int dtype, double *nu2_out, void *workspace, size_t ws_bytes,
                                   hd_stream_t stream)
{
    if (dtype != HD_U8 && dtype != HD_U16) return HD_ERR_DTYPE;
    if (H < 1 || W < 1) return HD_ERR_ARG;
    if (H > HD_DIM_MAX || W > HD_DIM_MAX) return HD_ERR_OVERFLOW;
    if (!f || !ref || !nu2_out || ((uintptr_t)nu2_out & 7)) return HD_ERR_ARG;
    const size_t es = dtype == HD_U8 ? 1 : 2;
    if (f_pitch < (size_t)W * es || ref_pitch < (size_t)W * es) return HD_ERR_ARG;
    if (es == 2 && (((uintptr_t)f | (uintptr_t)ref | f_pitch | ref_pitch) & 1)) return HD_ERR_ARG;
    if (!workspace || ((uintptr_t)workspace & 255) || ws_bytes < HD_REFNOISE_WORKSPACE_BYTES)
        return HD_ERR_WORKSPACE;
    RnParams p;
    p.f = static_cast<const uint8_t *>(f);
    p.r = static_cast<const uint8_t *>(ref);
    p.fp = (long long)f_pitch;
    p.rp = (long long)ref_pitch;
    p.H = (u32)H;
    p.W = (u32)W;
    p.elem = (int)es;
    p.out = nu2_out;
    p.ctl = static_cast<RnCtl *>(workspace);
    const int sms = sm_count();
    if (sms < 1) return HD_ERR_CUDA;
    const int grid = std::max(1, std::min(H, 2 * sms));
    if (es == 1) refnoise_kernel<1><<<grid, kRnThreads, 0, (cudaStream_t)stream>>>(p);
    else refnoise_kernel<2><<<grid, kRnThreads, 0, (cudaStream_t)stream>>>(p);
    if (cudaGetLastError() != cudaSuccess) return HD_ERR_CUDA;
    return HD_OK;
}

}  // extern "C"
