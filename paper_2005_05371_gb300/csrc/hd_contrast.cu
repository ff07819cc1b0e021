// hd_contrast.cu -- contrast stretch (Algorithm 1, step 4e) in one launch.
//
// The paper names the post-processing stretch and gives no rule.  The
// library reads it as a linear stretch between two saturation limits taken
// from the image histogram, at most k pixels saturating at each end:
//   k  = floor(fl64(tol * N)),  N = H * W,  0 <= tol < 1/2,
//   lo = the k-th smallest value (from 0), hi = the k-th largest,
//   out = x where lo == hi, else
//   out = floor((clamp(x, lo, hi) - lo) * maxv / (hi - lo) + 1/2)   (exact integers).
//
// One cooperative launch of a grid of one 1024-thread CTA per SM at most (all
// resident at once; the occupancy query sizes it).  Every CTA owns a fixed 1/gridDim share of the pixels in
// row-major order and makes three passes over it:
//   A  histogram of the share.  Up to 12 bits it lives in shared memory in R
//      interleaved copies (R = 32 for 8 bits, 2 for 12; lane l adds to copy
//      l mod R, so lanes with equal values do not collide); for 8-bit pixels
//      each thread first merges runs of equal values among its own pixels.  The copies are
//      then summed and added to the global histogram in the workspace.  13 to
//      16 bits add to the global histogram directly.  A release add on
//      `flushed` publishes the share;
//   B  one thread waits (bounded) until every CTA has flushed; then each warp
//      sums a sixteenth of the global histogram with coalesced loads, and the
//      warps whose range holds the k-th smallest or k-th largest value rescan
//      it with warp prefix sums to find lo and hi.  Up to 12 bits the CTA then
//      tabulates the map for every value in shared memory;
//   C  remap of the share, src -> dst (src == dst is allowed: every pixel is
//      read before it is written, by the thread that writes it, and pass C
//      starts only after every CTA has finished pass A).
// Tight images (pitch = row bytes, src and dst at the same 16-byte phase) are
// walked as one flat array with 16-byte vector loads and stores and scalar
// head and tail pieces; other pitches go row piece by row piece, pixel by
// pixel.
// The last CTA to finish pass B zeroes the histogram and the counters, so the
// workspace is zero again for the next call.  A wait that runs out latches
// DEVERR_TIMEOUT in this file's error word and skips the CTA's remap.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>
#include <vector>

#include "hd_contrast.h"
#include "hd_internal.h"
#include "hybrid_denoise.h"

namespace hd {
namespace {

typedef unsigned int u32;
typedef unsigned long long u64;

constexpr int kCsThreads = 1024;
constexpr int kCsWarps = kCsThreads / 32;
constexpr u32 kCsSharedBins = 4096;     // histograms of up to 12 bits live in shared memory
constexpr u32 kCsSharedWords = 8192;    // bins x copies of the shared histogram (32 KB)
constexpr int kCsMaxCtasPerSm = 1;
constexpr u32 kCsMinPxPerCta = kCsThreads * 16;
constexpr size_t kCsCtlBytes = 256;
constexpr u32 kFull = 0xffffffffu;

__device__ unsigned int g_contrast_error;

struct CsCtl {
    u32 flushed;      // CTAs whose share is in the global histogram
    u32 scanned;      // CTAs done with the global histogram
    u32 pad[62];
};
static_assert(sizeof(CsCtl) == kCsCtlBytes, "CsCtl layout");

struct CsParams {
    const uint8_t *src;
    uint8_t *dst;
    long long sp, dp;         // pitches, bytes
    u32 H, W, N;
    u32 maxv, nbins;          // 2^bits - 1, 2^bits
    u32 t_lo, t_hi;           // k + 1 and N - k: lo, hi are the first values whose
                              // cumulative count reaches them
    u32 *hist;                // nbins counters, zero before the launch
    CsCtl *ctl;
    u64 spin_limit;
    int flat;                 // walk src and dst as flat arrays (vector path)
    int shared;               // histogram and map table in shared memory
    u32 rshift;               // log2 of the shared histogram's copies (0 without)
};

__device__ __forceinline__ u32 ld_acquire(const u32 *p)
{
    u32 v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <int ES>
__device__ __forceinline__ u32 load_px(const uint8_t *base, u32 j)
{
    return ES == 1 ? (u32)base[j] : (u32) reinterpret_cast<const uint16_t *>(base)[j];
}

template <int ES>
__device__ __forceinline__ void store_px(uint8_t *base, u32 j, u32 v)
{
    if (ES == 1) base[j] = (uint8_t)v;
    else reinterpret_cast<uint16_t *>(base)[j] = (uint16_t)v;
}

// The 16 / ES pixels of a 16-byte vector, first pixel at the lowest address.
template <int ES>
__device__ __forceinline__ void unpack(const uint4 &v, u32 (&px)[16 / ES])
{
    const u32 w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 16 / ES; ++i)
        px[i] = ES == 1 ? (w[i >> 2] >> (8 * (i & 3))) & 0xffu : (w[i >> 1] >> (16 * (i & 1))) & 0xffffu;
}

template <int ES>
__device__ __forceinline__ uint4 pack(const u32 (&px)[16 / ES])
{
    u32 w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int i = 0; i < 16 / ES; ++i) w[ES == 1 ? i >> 2 : i >> 1] |= px[i] << (ES == 1 ? 8 * (i & 3) : 16 * (i & 1));
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// Add cnt to bin v: copy (lane mod R) of the shared histogram, or the global one.
__device__ __forceinline__ void hadd(u32 *h, u32 rshift, u32 lane, u32 v, u32 cnt)
{
    atomicAdd(h + ((v << rshift) | (lane & ((1u << rshift) - 1u))), cnt);
}

// round-half-up((c - lo) maxv / q) for c = clamp(x, lo, hi), q = hi - lo > 0.
// The binary32 estimate floor(c * fl(maxv / q) + 1/2) is within 0.01 of the
// exact value for c, maxv < 2^16, so one step by the exact remainder of
// 2 c maxv + q over 2 q (32 x 32 -> 64-bit products) corrects it.
__device__ __forceinline__ u32 stretch_px(u32 x, u32 lo, u32 hi, u32 maxv, float scale)
{
    const u32 c = min(max(x, lo), hi) - lo;
    const u32 q = hi - lo;
    u32 est = __float2uint_rz(__fmaf_rn((float)c, scale, 0.5f));
    const long long r = 2ll * ((long long)c * (long long)maxv) + (long long)q - 2ll * ((long long)est * (long long)q);
    if (r < 0) --est;
    else if (r >= 2ll * (long long)q) ++est;
    return est;
}

// Walk the share [b0, b1) one row piece at a time; f(src row piece, dst row
// piece, pixels in the piece).  Every thread of the CTA runs the same iterations.
template <class F>
__device__ __forceinline__ void for_pieces(const CsParams &p, int es, u32 b0, u32 b1, F f)
{
    u32 i = b0;
    while (i < b1) {
        const u32 y = i / p.W;
        const u32 x0 = i - y * p.W;
        const u32 n = min(p.W - x0, b1 - i);
        f(p.src + (long long)y * p.sp + (long long)x0 * es, p.dst + (long long)y * p.dp + (long long)x0 * es, n);
        i += n;
    }
}

// The flat share [b0, b1): scalar pixels before the first and after the last
// 16-byte boundary of src, and nvec whole vectors between them.
struct FlatSplit {
    u32 head, nvec, tail;     // pixels, vectors, pixels
};

template <int ES>
__device__ __forceinline__ FlatSplit flat_split(const CsParams &p, u32 b0, u32 b1)
{
    const uintptr_t a0 = reinterpret_cast<uintptr_t>(p.src) + (uintptr_t)b0 * ES;
    const u32 bytes = (b1 - b0) * ES;
    const u32 hb = min(bytes, (u32)((16u - (a0 & 15u)) & 15u));
    FlatSplit f;
    f.head = hb / ES;
    f.nvec = (bytes - hb) >> 4;
    f.tail = (bytes - hb - (f.nvec << 4)) / ES;
    return f;
}

// Lowest bin whose cumulative count reaches T, for the warp whose bin range
// [wb0, wb1) holds it (pre = pixels in bins below wb0).  Warp-uniform.
__device__ __forceinline__ void warp_find(const u32 *hist, u32 wb0, u32 wb1, u32 pre, u32 T, u32 lane, u32 *out)
{
    u32 c = pre;
    for (u32 b = wb0; b < wb1; b += 32) {
        const u32 bin = b + lane;
        u32 incl = bin < wb1 ? __ldcg(hist + bin) : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u32 t = __shfl_up_sync(kFull, incl, o);
            if (lane >= (u32)o) incl += t;
        }
        const u32 hit = __ballot_sync(kFull, c + incl >= T);
        if (hit) {
            if (lane == (u32)(__ffs(hit) - 1)) *out = bin;
            return;
        }
        c += __shfl_sync(kFull, incl, 31);
    }
}

// Index of the first of four bins whose cumulative count, from `pre`, reaches T.
__device__ __forceinline__ u32 first_reaching(const u32 (&c4)[4], u32 pre, u32 T)
{
    u32 c = pre, idx = 3;
    bool found = false;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        c += c4[j];
        if (!found && c >= T) {
            idx = (u32)j;
            found = true;
        }
    }
    return idx;
}

template <int ES>
__global__ void __launch_bounds__(kCsThreads, 1) contrast_kernel(CsParams p)
{
    extern __shared__ u32 sh[];
    __shared__ u32 s_wsum[kCsWarps];
    __shared__ u32 s_lo, s_hi;
    __shared__ int s_ok, s_last;
    constexpr int V = 16 / ES;                // pixels in a 16-byte vector
    const u32 tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const u32 rshift = p.rshift;
    u32 *h = p.shared ? sh : p.hist;
    uint16_t *lut = reinterpret_cast<uint16_t *>(sh + (p.shared ? (p.nbins << rshift) : 0u));
    if (p.shared)
        for (u32 b = tid; b < (p.nbins << rshift); b += kCsThreads) sh[b] = 0;
    if (tid == 0) {
        s_lo = 0;
        s_hi = 0;
    }
    __syncthreads();

    const u32 b0 = (u32)((u64)p.N * blockIdx.x / gridDim.x);
    const u32 b1 = (u32)((u64)p.N * (blockIdx.x + 1) / gridDim.x);

    // ---- pass A: histogram of the share
    if (p.flat) {
        const FlatSplit f = flat_split<ES>(p, b0, b1);
        if (tid < f.head) hadd(h, rshift, lane, min(load_px<ES>(p.src, b0 + tid), p.maxv), 1u);
        if (tid < f.tail) hadd(h, rshift, lane, min(load_px<ES>(p.src, b1 - f.tail + tid), p.maxv), 1u);
        const uint4 *vs = reinterpret_cast<const uint4 *>(p.src + (size_t)(b0 + f.head) * ES);
        for (u32 c0 = tid; c0 < f.nvec; c0 += 4 * kCsThreads) {
            uint4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const u32 c = c0 + u * kCsThreads;
                if (c < f.nvec) v[u] = vs[c];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (c0 + u * kCsThreads >= f.nvec) break;
                u32 px[V];
                unpack<ES>(v[u], px);
                if (ES == 1) {
                    // 8-bit: runs of equal values among this thread's pixels add once
                    u32 cur = px[0], cnt = 1;
#pragma unroll
                    for (int i = 1; i < V; ++i) {
                        if (px[i] == cur) {
                            ++cnt;
                        } else {
                            hadd(h, rshift, lane, cur, cnt);
                            cur = px[i];
                            cnt = 1;
                        }
                    }
                    hadd(h, rshift, lane, cur, cnt);
                } else {
#pragma unroll
                    for (int i = 0; i < V; ++i) hadd(h, rshift, lane, min(px[i], p.maxv), 1u);
                }
            }
        }
    } else {
        for_pieces(p, ES, b0, b1, [&](const uint8_t *srow, uint8_t *, u32 n) {
            for (u32 j = tid; j < n; j += kCsThreads) hadd(h, rshift, lane, min(load_px<ES>(srow, j), p.maxv), 1u);
        });
    }
    if (p.shared) {
        __syncthreads();
        const u32 R = 1u << rshift;
        for (u32 b = tid; b < p.nbins; b += kCsThreads) {
            u32 c = 0;
            for (u32 r = 0; r < R; ++r) c += sh[(b << rshift) | ((r + lane) & (R - 1u))];
            if (c) atomicAdd(p.hist + b, c);
        }
    }
    __syncthreads();

    // ---- pass B: wait for every share, then find lo and hi
    if (tid == 0) {
        __threadfence();
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&p.ctl->flushed) : "memory");
        int ok = 1;
        u64 polls = 0;
        while (ld_acquire(&p.ctl->flushed) < gridDim.x) {
            if (++polls > p.spin_limit) {
                atomicOr(&g_contrast_error, DEVERR_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(polls < 64 ? 32 : 256);
        }
        s_ok = ok;
    }
    __syncthreads();
    if (s_ok) {
        if (p.nbins <= 4u * kCsThreads) {
            // four bins a thread, one coalesced read, block prefix sums
            const u32 b4 = 4u * tid;
            u32 c4[4] = {0u, 0u, 0u, 0u};
            if (b4 < p.nbins) {
                const uint4 v = __ldcg(reinterpret_cast<const uint4 *>(p.hist) + tid);
                c4[0] = v.x;
                c4[1] = b4 + 1 < p.nbins ? v.y : 0u;
                c4[2] = b4 + 2 < p.nbins ? v.z : 0u;
                c4[3] = b4 + 3 < p.nbins ? v.w : 0u;
            }
            const u32 cnt = c4[0] + c4[1] + c4[2] + c4[3];
            u32 incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const u32 t = __shfl_up_sync(kFull, incl, o);
                if (lane >= (u32)o) incl += t;
            }
            if (lane == 31) s_wsum[warp] = incl;
            __syncthreads();
            if (warp == 0) {
                u32 t = s_wsum[lane];
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const u32 u = __shfl_up_sync(kFull, t, o);
                    if (lane >= (u32)o) t += u;
                }
                s_wsum[lane] = t;
            }
            __syncthreads();
            const u32 pre = (warp ? s_wsum[warp - 1] : 0u) + incl - cnt;   // pixels in bins below b4
            if (pre < p.t_lo && p.t_lo <= pre + cnt) s_lo = b4 + first_reaching(c4, pre, p.t_lo);
            if (pre < p.t_hi && p.t_hi <= pre + cnt) s_hi = b4 + first_reaching(c4, pre, p.t_hi);
        } else {
            // 13..16 bits: each warp sums its range, then rescans the range
            // that holds the limit
            const u32 wb0 = (u32)((u64)warp * p.nbins / kCsWarps), wb1 = (u32)((u64)(warp + 1) * p.nbins / kCsWarps);
            u32 sum = 0;
            for (u32 b = wb0 + lane; b < wb1; b += 32) sum += __ldcg(p.hist + b);
            sum = __reduce_add_sync(kFull, sum);
            if (lane == 0) s_wsum[warp] = sum;
            __syncthreads();
            u32 pre = 0;
            for (u32 w = 0; w < warp; ++w) pre += s_wsum[w];
            if (pre < p.t_lo && p.t_lo <= pre + sum) warp_find(p.hist, wb0, wb1, pre, p.t_lo, lane, &s_lo);
            if (pre < p.t_hi && p.t_hi <= pre + sum) warp_find(p.hist, wb0, wb1, pre, p.t_hi, lane, &s_hi);
        }
    }
    __syncthreads();
    // count this CTA out of the histogram; the result is needed only at the
    // end, so the round trip overlaps the remap
    u32 old_scanned = 0;
    if (tid == 0) {
        __threadfence();
        old_scanned = atomicAdd(&p.ctl->scanned, 1u);
    }

    // ---- pass C: remap the share (nothing to do after a timeout, or for the
    // identity in place)
    const u32 lo = s_lo, hi = s_hi;
    if (s_ok && !(lo == hi && p.src == p.dst && p.sp == p.dp)) {
        const float scale = lo < hi ? __fdiv_rn((float)p.maxv, (float)(hi - lo)) : 0.0f;
        if (p.shared) {
            for (u32 v = tid; v < p.nbins; v += kCsThreads) lut[v] = (uint16_t)(lo < hi ? stretch_px(v, lo, hi, p.maxv, scale) : v);
            __syncthreads();
        }
        auto map = [&](u32 x) -> u32 {
            if (p.shared) return lut[min(x, p.maxv)];
            return lo < hi ? stretch_px(x, lo, hi, p.maxv, scale) : x;
        };
        if (p.flat) {
            const FlatSplit f = flat_split<ES>(p, b0, b1);
            if (tid < f.head) store_px<ES>(p.dst, b0 + tid, map(load_px<ES>(p.src, b0 + tid)));
            if (tid < f.tail) store_px<ES>(p.dst, b1 - f.tail + tid, map(load_px<ES>(p.src, b1 - f.tail + tid)));
            const uint4 *vs = reinterpret_cast<const uint4 *>(p.src + (size_t)(b0 + f.head) * ES);
            uint4 *vd = reinterpret_cast<uint4 *>(p.dst + (size_t)(b0 + f.head) * ES);
            for (u32 c0 = tid; c0 < f.nvec; c0 += 4 * kCsThreads) {
                uint4 v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const u32 c = c0 + u * kCsThreads;
                    if (c < f.nvec) v[u] = vs[c];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const u32 c = c0 + u * kCsThreads;
                    if (c >= f.nvec) break;
                    u32 px[V];
                    unpack<ES>(v[u], px);
#pragma unroll
                    for (int i = 0; i < V; ++i) px[i] = map(px[i]);
                    vd[c] = pack<ES>(px);
                }
            }
        } else {
            for_pieces(p, ES, b0, b1, [&](const uint8_t *srow, uint8_t *drow, u32 n) {
                for (u32 j = tid; j < n; j += kCsThreads) store_px<ES>(drow, j, map(load_px<ES>(srow, j)));
            });
        }
    }

    // the last CTA out of the histogram clears it and the counters
    if (tid == 0) {
        __threadfence();
        s_last = old_scanned == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
        for (u32 b = tid; b < p.nbins; b += kCsThreads) p.hist[b] = 0;
        __syncthreads();
        if (tid == 0) {
            p.ctl->flushed = 0;
            p.ctl->scanned = 0;
            __threadfence();
        }
    }
}

inline size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

size_t hist_bytes(int bits) { return round_up(((size_t)1 << bits) * sizeof(u32), 256); }

// Resident CTAs per SM at the largest shared-memory size a launch uses
// (a lower bound for every smaller size), per device and element size.
int contrast_ctas_per_sm(int es)
{
    static std::mutex mu;
    static std::vector<int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    const int slot = 2 * dev + (es == 2 ? 1 : 0);
    std::lock_guard<std::mutex> lk(mu);
    if ((int)cache.size() <= slot) cache.resize(slot + 1, -1);
    if (cache[slot] < 0) {
        const size_t smem = kCsSharedWords * sizeof(u32) + kCsSharedBins * sizeof(uint16_t);
        int n = 0;
        const cudaError_t e = es == 1
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, contrast_kernel<1>, kCsThreads, smem)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, contrast_kernel<2>, kCsThreads, smem);
        if (e != cudaSuccess) return 0;
        cache[slot] = n;
    }
    return cache[slot];
}

hd_status check_contrast(const hd_image *img, double tol)
{
    if (!img) return HD_ERR_ARG;
    if (img->dtype != HD_U8 && img->dtype != HD_U16) return HD_ERR_DTYPE;
    if (img->dtype == HD_U8 && img->p.bits != 8) return HD_ERR_DTYPE;
    if (img->dtype == HD_U16 && (img->p.bits < 1 || img->p.bits > 16)) return HD_ERR_DTYPE;
    if (img->H < 1 || img->W < 1) return HD_ERR_ARG;
    if (img->H > HD_DIM_MAX || img->W > HD_DIM_MAX) return HD_ERR_OVERFLOW;
    if (!img->src || !img->dst) return HD_ERR_ARG;
    if (!(tol >= 0.0 && tol < 0.5)) return HD_ERR_ARG;
    const size_t es = img->dtype == HD_U8 ? 1 : 2;
    const size_t row = (size_t)img->W * es;
    if (img->src_pitch < row || img->dst_pitch < row) return HD_ERR_ARG;
    if (es == 2) {
        if ((img->src_pitch | img->dst_pitch) & 1) return HD_ERR_ARG;
        if (((uintptr_t)img->src | (uintptr_t)img->dst) & 1) return HD_ERR_ARG;
    }
    // in place (the same buffer and pitch) or no overlap at all
    if (img->src == img->dst) return img->src_pitch == img->dst_pitch ? HD_OK : HD_ERR_ARG;
    const uintptr_t s0 = (uintptr_t)img->src, s1 = s0 + (size_t)(img->H - 1) * img->src_pitch + row;
    const uintptr_t d0 = (uintptr_t)img->dst, d1 = d0 + (size_t)(img->H - 1) * img->dst_pitch + row;
    if (s0 < d1 && d0 < s1) return HD_ERR_ARG;
    return HD_OK;
}

}  // namespace

int read_and_clear_contrast_error(unsigned int *out)
{
    unsigned int v = 0, zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_contrast_error, sizeof(v));
    if (e == cudaSuccess && v) e = cudaMemcpyToSymbol(g_contrast_error, &zero, sizeof(zero));
    *out = v;
    return (int)e;
}

}  // namespace hd

using namespace hd;

extern "C" {

hd_status contrast_workspace_size(int H, int W, int dtype, const hd_params *p, size_t *bytes)
{
    if (!p || !bytes) return HD_ERR_ARG;
    if (dtype != HD_U8 && dtype != HD_U16) return HD_ERR_DTYPE;
    if ((dtype == HD_U8 && p->bits != 8) || p->bits < 1 || p->bits > 16) return HD_ERR_DTYPE;
    if (H < 1 || W < 1) return HD_ERR_ARG;
    if (H > HD_DIM_MAX || W > HD_DIM_MAX) return HD_ERR_OVERFLOW;
    *bytes = kCsCtlBytes + hist_bytes(p->bits);
    return HD_OK;
}

hd_status contrast_stretch(const hd_image *img, double tol, void *workspace, size_t ws_bytes,
                           hd_stream_t stream)
{
    hd_status st = check_contrast(img, tol);
    if (st != HD_OK) return st;
    size_t need = 0;
    st = contrast_workspace_size(img->H, img->W, img->dtype, &img->p, &need);
    if (st != HD_OK) return st;
    if (!workspace || ((uintptr_t)workspace & 255) || ws_bytes < need) return HD_ERR_WORKSPACE;

    CsParams p;
    p.src = static_cast<const uint8_t *>(img->src);
    p.dst = static_cast<uint8_t *>(img->dst);
    p.sp = (long long)img->src_pitch;
    p.dp = (long long)img->dst_pitch;
    p.H = (u32)img->H;
    p.W = (u32)img->W;
    p.N = p.H * p.W;                      // <= 65535^2 < 2^32
    const int es = img->dtype == HD_U8 ? 1 : 2;
    p.nbins = 1u << img->p.bits;
    p.maxv = p.nbins - 1;
    const u64 k = (u64)std::floor(tol * (double)p.N);
    p.t_lo = (u32)(k + 1);
    p.t_hi = (u32)(p.N - k);
    p.ctl = static_cast<CsCtl *>(workspace);
    p.hist = reinterpret_cast<u32 *>(static_cast<uint8_t *>(workspace) + kCsCtlBytes);
    p.spin_limit = spin_limit_polls();

    // vector path: both images tight (or one row) and at the same 16-byte phase
    const size_t row = (size_t)img->W * es;
    p.flat = (img->H == 1 || (img->src_pitch == row && img->dst_pitch == row)) &&
             (((uintptr_t)img->src - (uintptr_t)img->dst) & 15) == 0;
    p.shared = p.nbins <= kCsSharedBins;
    p.rshift = 0;
    if (p.shared)
        while ((p.nbins << (p.rshift + 1)) <= kCsSharedWords && p.rshift < 5) ++p.rshift;
    const size_t smem = p.shared ? (size_t)(p.nbins << p.rshift) * sizeof(u32) + (size_t)p.nbins * sizeof(uint16_t)
                                 : 0;
    const int per_sm = std::min(contrast_ctas_per_sm(es), kCsMaxCtasPerSm);
    const int sms = sm_count();
    if (per_sm < 1 || sms < 1) return HD_ERR_CUDA;
    const u32 by_size = (p.N + kCsMinPxPerCta - 1) / kCsMinPxPerCta;
    const int grid = (int)std::max(1u, std::min(by_size, (u32)(sms * per_sm)));
    // a cooperative launch: the CTAs wait for one another, so they must all be
    // resident at once (the bounded wait stays as a safety net)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kCsThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = (cudaStream_t)stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const cudaError_t e = es == 1 ? cudaLaunchKernelEx(&cfg, contrast_kernel<1>, p)
                                  : cudaLaunchKernelEx(&cfg, contrast_kernel<2>, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return HD_ERR_CUDA;
    }
    return HD_OK;
}

}  // extern "C"
