// hd_kernel.cu -- the persistent hybrid-denoise kernel for sm_103a.
//
// One launch runs a whole image (or a batch of images) through
//   phase 1: adaptive median (Algorithm 1, step 6) on a shared-memory tile
//            plus the Wiener halo, then the exact local statistics D of the
//            median output and a per-image integer sum of D (the noise
//            variance of the Wiener stage is the mean local variance);
//   phase 2: Wiener apply (Algorithm 1, step 4d) once every phase-1 tile of
//            that image is done.
// Work items (image, phase, tile) are handed out in ticket order by one
// global counter.  A CTA takes its next ticket only after any wait of its
// current item is over, so every wait is on items held by running CTAs.
// Waits are bounded: after lp.spin_limit polls the CTA latches
// DEVERR_TIMEOUT in g_device_error and skips the item.
//
// Median: 3x3 window statistics for every pixel from row-sorted triples
// (median of nine = med3(max of row minima, med3 of row medians, min of row
// maxima)); pixels failing level A join a shared-memory worklist that is
// re-compacted for every larger window k = 5..Smax and resolved one warp per
// pixel with a bitwise radix select over the k*k samples.
//
// Wiener: S1 = sum f and S2 = sum f^2 over w x w by separable sums in
// shared memory, exact in 32/64-bit integers; D = n*S2 - S1^2 exact.  The gain
// and output use binary32 with a fixed order of correctly rounded operations
// (no contraction):
//   mu  = fl(S1) * fl(1/n)            s2 = fl(D) * fl(1/n^2)      v2 = fl(nu2)
//   den = max(s2, v2)                 num = max(s2 - v2, 0)
//   y   = den > 0 ? mu + (num / den) * (fl(f) - mu) : mu
//   out = min(maxv, floor(y + 0.5))
// nu2 = fl64( fl64(sum D) / (n*n*H*W) ) with a correctly rounded 128-bit to
// binary64 conversion; binary64 is used only for this one scalar per image.
#include <cuda_runtime.h>
#include <cstdint>
#include "hd_internal.h"

namespace hd {

__device__ unsigned int g_device_error;

namespace {

struct Smem {
    unsigned long long *V2;   // [tile_h][FWmax] vertical sums of f^2
    unsigned int *V1;         // [tile_h][FWmax] vertical sums of f
    unsigned int *wl0;        // worklists of (row << 16 | col) in the f region
    unsigned int *wl1;
    unsigned short *gs;       // noisy input region (f region + median halo)
    unsigned short *fs;       // median output region (tile + Wiener halo)
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

struct SmemLayout {
    size_t v2, v1, wl0, wl1, gs, fs, total;
};

__host__ __device__ inline SmemLayout layout(int tile_w, int tile_h, int ra_max, int rw_max)
{
    const size_t FW = tile_w + 2 * rw_max, FH = tile_h + 2 * rw_max;
    const size_t GW = FW + 2 * ra_max, GH = FH + 2 * ra_max;
    SmemLayout L;
    size_t off = 0;
    L.v2 = off;  off = align16(off + sizeof(unsigned long long) * tile_h * FW);
    L.v1 = off;  off = align16(off + sizeof(unsigned int) * tile_h * FW);
    L.wl0 = off; off = align16(off + sizeof(unsigned int) * FH * FW);
    L.wl1 = off; off = align16(off + sizeof(unsigned int) * FH * FW);
    L.gs = off;  off = align16(off + sizeof(unsigned short) * GH * GW);
    L.fs = off;  off = align16(off + sizeof(unsigned short) * FH * FW);
    L.total = off;
    return L;
}

// Half-sample symmetric extension with period 2n, valid for any i.
__device__ __forceinline__ int refl(int i, int n)
{
    if ((unsigned)i < (unsigned)n) return i;
    const int p = 2 * n;
    int m = i % p;
    if (m < 0) m += p;
    return m < n ? m : p - 1 - m;
}

__device__ __forceinline__ unsigned umin(unsigned a, unsigned b) { return a < b ? a : b; }
__device__ __forceinline__ unsigned umax(unsigned a, unsigned b) { return a > b ? a : b; }

// Sort three values: on return a <= b <= c.
__device__ __forceinline__ void sort3(unsigned &a, unsigned &b, unsigned &c)
{
    unsigned lo = umin(a, b), hi = umax(a, b);
    unsigned lo2 = umin(lo, c), t = umax(lo, c);
    a = lo2;
    b = umin(hi, t);
    c = umax(hi, t);
}

__device__ __forceinline__ unsigned med3(unsigned a, unsigned b, unsigned c)
{
    return umax(umin(a, b), umin(umax(a, b), c));
}

__device__ __forceinline__ unsigned load_px(const uint8_t *base, long long pitch, int elem, int y, int x,
                                            bool cg)
{
    const uint8_t *row = base + (long long)y * pitch;
    if (elem == 1) return cg ? (unsigned)__ldcg(row + x) : (unsigned)row[x];
    const unsigned short *r16 = reinterpret_cast<const unsigned short *>(row);
    return cg ? (unsigned)__ldcg(r16 + x) : (unsigned)r16[x];
}

// Copy image rows [y0, y0+SH) x cols [x0, x0+SW) into shared memory (stride
// SW), reflecting out-of-range indices or reading zeros there.
__device__ void load_region(unsigned short *dst, int SW, int SH, const uint8_t *base, long long pitch,
                            int elem, int H, int W, int y0, int x0, bool zero_outside, bool cg)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int ry = warp; ry < SH; ry += kThreads / 32) {
        const int gy = y0 + ry;
        const bool yout = (unsigned)gy >= (unsigned)H;
        const int sy = refl(gy, H);
        for (int rx = lane; rx < SW; rx += 32) {
            const int gx = x0 + rx;
            unsigned v;
            if (zero_outside && (yout || (unsigned)gx >= (unsigned)W)) v = 0;
            else v = load_px(base, pitch, elem, sy, refl(gx, W), cg);
            dst[ry * SW + rx] = (unsigned short)v;
        }
    }
}

struct WinStats {
    unsigned zmin, zmed, zmax;
};

// Order statistics of the k x k window centred at c (stride GW), one warp.
// The median is the (k*k-1)/2-th smallest sample, found bit by bit from the
// most significant bit where zmin and zmax differ.
__device__ WinStats warp_window_stats(const unsigned short *c, int GW, int k, int lane)
{
    const int r = k >> 1, cnt = k * k;
    const int nslots = (cnt + 31) >> 5;      // <= 8 for k <= 15
    unsigned v[8];
    unsigned lmin = 0xffffffffu, lmax = 0u;
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        unsigned x = 0xffffffffu;
        const int j = lane + 32 * s;
        if (s < nslots && j < cnt) {
            const int q = j / k;
            x = c[(q - r) * GW + (j - q * k - r)];
            lmin = umin(lmin, x);
            lmax = umax(lmax, x);
        }
        v[s] = x;
    }
    const unsigned zmin = __reduce_min_sync(0xffffffffu, lmin);
    const unsigned zmax = __reduce_max_sync(0xffffffffu, lmax);
    const unsigned diff = zmin ^ zmax;
    if (diff == 0) return {zmin, zmin, zmax};
    const int hb = 31 - __clz(diff);
    unsigned prefix = zmin & ~((2u << hb) - 1u);
    unsigned rank = (unsigned)(cnt - 1) >> 1;
    for (int b = hb; b >= 0; --b) {
        unsigned c0 = 0;
#pragma unroll
        for (int s = 0; s < 8; ++s)
            if (s < nslots) c0 += ((v[s] ^ prefix) >> b) == 0u;
        c0 = __reduce_add_sync(0xffffffffu, c0);
        if (rank >= c0) {
            rank -= c0;
            prefix |= 1u << b;
        }
    }
    return {zmin, prefix, zmax};
}

// Adaptive median over the f region (FW x FH) from the g region (stride GW,
// origin Ra rows/cols before the f region).  Writes fs.
__device__ void amf_region(const ImgDesc &d, const Smem &sm, int FW, int FH, int GW, int Ra, int *s_cnt)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int smax = d.smax;
    const bool keep = d.unresolved != 0;
    // --- k = 3 for every pixel
    for (int ry = warp; ry < FH; ry += kThreads / 32) {
        const unsigned short *grow = sm.gs + (ry + Ra) * GW + Ra;
        for (int rx0 = 0; rx0 < FW; rx0 += 32) {
            const int rx = rx0 + lane;
            bool grow_it = false;
            if (rx < FW) {
                const unsigned short *c = grow + rx;
                unsigned a0 = c[-GW - 1], a1 = c[-GW], a2 = c[-GW + 1];
                unsigned b0 = c[-1], b1 = c[0], b2 = c[1];
                unsigned e0 = c[GW - 1], e1 = c[GW], e2 = c[GW + 1];
                const unsigned zxy = b1;
                sort3(a0, a1, a2);
                sort3(b0, b1, b2);
                sort3(e0, e1, e2);
                const unsigned zmin = umin(umin(a0, b0), e0);
                const unsigned zmax = umax(umax(a2, b2), e2);
                const unsigned zmed = med3(umax(umax(a0, b0), e0), med3(a1, b1, e1),
                                           umin(umin(a2, b2), e2));
                unsigned out;
                if (zmin < zmed && zmed < zmax) {                  // level A
                    out = (zmin < zxy && zxy < zmax) ? zxy : zmed;  // level B
                } else if (smax == 3) {
                    out = keep ? zxy : zmed;
                } else {
                    out = zmed;
                    grow_it = true;
                }
                sm.fs[ry * FW + rx] = (unsigned short)out;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, grow_it);
            if (bal) {
                int base = 0;
                if (lane == 0) base = atomicAdd(&s_cnt[0], __popc(bal));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (grow_it)
                    sm.wl0[base + __popc(bal & ((1u << lane) - 1u))] = ((unsigned)ry << 16) | (unsigned)rx;
            }
        }
    }
    __syncthreads();
    // --- k = 5 .. Smax on the compacted worklist, one warp per pixel
    unsigned int *cur = sm.wl0, *nxt = sm.wl1;
    int ci = 0;
    for (int k = 5; k <= smax; k += 2) {
        const int n = s_cnt[ci];
        if (n == 0) break;
        if (threadIdx.x == 0) s_cnt[ci ^ 1] = 0;
        __syncthreads();
        for (int e = warp; e < n; e += kThreads / 32) {
            const unsigned ent = cur[e];
            const int ry = (int)(ent >> 16), rx = (int)(ent & 0xffffu);
            const unsigned short *c = sm.gs + (ry + Ra) * GW + (rx + Ra);
            const unsigned zxy = c[0];
            const WinStats st = warp_window_stats(c, GW, k, lane);
            if (lane == 0) {
                if (st.zmin < st.zmed && st.zmed < st.zmax) {
                    sm.fs[ry * FW + rx] = (unsigned short)((st.zmin < zxy && zxy < st.zmax) ? zxy : st.zmed);
                } else if (k == smax) {
                    sm.fs[ry * FW + rx] = (unsigned short)(keep ? zxy : st.zmed);
                } else {
                    const int p = atomicAdd(&s_cnt[ci ^ 1], 1);
                    nxt[p] = ent;
                }
            }
        }
        __syncthreads();
        unsigned int *t = cur; cur = nxt; nxt = t;
        ci ^= 1;
    }
}

// Vertical sums over w rows for output rows [0, th) of the f region.
__device__ void vertical_sums(const Smem &sm, int FW, int th, int w)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int SEG = 4;
    const int nseg = (th + SEG - 1) / SEG;
    const int ncc = (FW + 31) >> 5;
    for (int it = warp; it < nseg * ncc; it += kThreads / 32) {
        const int seg = it / ncc, cc = it - seg * ncc;
        const int c = cc * 32 + lane;
        if (c >= FW) continue;
        const int oy0 = seg * SEG, oy1 = min(th, oy0 + SEG);
        unsigned s1 = 0;
        unsigned long long s2 = 0;
        for (int dy = 0; dy < w; ++dy) {
            const unsigned v = sm.fs[(oy0 + dy) * FW + c];
            s1 += v;
            s2 += (unsigned long long)(v * v);
        }
        sm.V1[oy0 * FW + c] = s1;
        sm.V2[oy0 * FW + c] = s2;
        for (int oy = oy0 + 1; oy < oy1; ++oy) {
            const unsigned vin = sm.fs[(oy + w - 1) * FW + c];
            const unsigned vout = sm.fs[(oy - 1) * FW + c];
            s1 += vin - vout;
            s2 += (unsigned long long)(vin * vin);
            s2 -= (unsigned long long)(vout * vout);
            sm.V1[oy * FW + c] = s1;
            sm.V2[oy * FW + c] = s2;
        }
    }
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    return x;
}

// Correctly rounded conversion of hi*2^64 + lo to binary64.
__device__ double u128_to_double(unsigned long long hi, unsigned long long lo)
{
    if (hi == 0) return __ull2double_rn(lo);
    const int s = __clzll((long long)hi);
    unsigned long long top = s == 0 ? hi : ((hi << s) | (lo >> (64 - s)));
    const unsigned long long rest = lo << s;
    top |= (rest != 0ull) ? 1ull : 0ull;    // sticky bit, far below the rounding position
    return scalbn(__ull2double_rn(top), 64 - s);
}

__device__ bool wait_phase1(const ImgDesc &d, unsigned total, unsigned long long limit, int *s_flag)
{
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned long long polls = 0;
        volatile unsigned int *cnt = &d.ctl->p1_done;
        while (*cnt < total) {
            if (++polls > limit) {
                atomicOr(&g_device_error, DEVERR_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(polls < 64 ? 32 : 256);
        }
        __threadfence();
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

struct BlockShared {
    int item[2];
    int cnt[2];
    int flag;
    unsigned long long red[kThreads / 32];
};

__device__ void run_item(const ImgDesc &d, int phase, int tile, const LaunchParams &lp, const Smem &sm,
                         BlockShared &bs, int nextbuf, bool &prefetched)
{
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int tyi = tile / d.tiles_x, txi = tile - tyi * d.tiles_x;
    const int x0 = txi * lp.tile_w, y0 = tyi * lp.tile_h;
    const int tw = min(lp.tile_w, d.W - x0), th = min(lp.tile_h, d.H - y0);
    const int mode = d.mode;
    const bool two_phase = (mode == MODE_WIENER_EST || mode == MODE_HYBRID_EST);
    const bool do_amf = phase == 1 && (mode == MODE_AMF || mode == MODE_HYBRID_EST || mode == MODE_HYBRID_GIVEN);
    const int Rw = mode == MODE_AMF ? 0 : (d.w >> 1);
    const int Ra = do_amf ? (d.smax >> 1) : 0;
    const int FW = tw + 2 * Rw, FH = th + 2 * Rw;

    if (phase == 2) {
        const unsigned total = (unsigned)(d.tiles_x * d.tiles_y);
        const bool ok = wait_phase1(d, total, lp.spin_limit, &bs.flag);
        if (tid == 0 && lp.ticket) bs.item[nextbuf] = (int)atomicAdd(lp.ticket, 1u);
        prefetched = true;
        if (!ok) return;
    }

    // ---- fill the f region in shared memory
    if (do_amf) {
        const int GW = FW + 2 * Ra, GH = FH + 2 * Ra;
        if (tid == 0) bs.cnt[0] = 0;
        load_region(sm.gs, GW, GH, d.src, d.src_pitch, d.elem, d.H, d.W, y0 - Rw - Ra, x0 - Rw - Ra,
                    false, false);
        __syncthreads();
        amf_region(d, sm, FW, FH, GW, Ra, bs.cnt);
        __syncthreads();
        if (Rw > 0 && d.border_zero) {
            // zero-border Wiener: samples outside the image read 0
            for (int i = tid; i < FW * FH; i += kThreads) {
                const int ry = i / FW, rx = i - ry * FW;
                const int gy = y0 - Rw + ry, gx = x0 - Rw + rx;
                if ((unsigned)gy >= (unsigned)d.H || (unsigned)gx >= (unsigned)d.W) sm.fs[i] = 0;
            }
            __syncthreads();
        }
    } else {
        const bool from_f = (phase == 2 && mode == MODE_HYBRID_EST);
        load_region(sm.fs, FW, FH, from_f ? d.fbuf : d.src, from_f ? d.f_pitch : d.src_pitch, d.elem,
                    d.H, d.W, y0 - Rw, x0 - Rw, d.border_zero != 0, from_f);
        __syncthreads();
    }

    // ---- median only: store and finish
    if (mode == MODE_AMF) {
        for (int oy = warp; oy < th; oy += kThreads / 32) {
            uint8_t *row = d.dst + (long long)(y0 + oy) * d.dst_pitch;
            for (int ox = lane; ox < tw; ox += 32) {
                const unsigned v = sm.fs[oy * FW + ox];
                if (d.elem == 1) row[x0 + ox] = (uint8_t)v;
                else reinterpret_cast<unsigned short *>(row)[x0 + ox] = (unsigned short)v;
            }
        }
        return;
    }

    // ---- phase 1 of the hybrid keeps the median output for phase 2
    if (phase == 1 && mode == MODE_HYBRID_EST) {
        for (int oy = warp; oy < th; oy += kThreads / 32) {
            uint8_t *row = d.fbuf + (long long)(y0 + oy) * d.f_pitch;
            for (int ox = lane; ox < tw; ox += 32) {
                const unsigned v = sm.fs[(oy + Rw) * FW + ox + Rw];
                if (d.elem == 1) row[x0 + ox] = (uint8_t)v;
                else reinterpret_cast<unsigned short *>(row)[x0 + ox] = (unsigned short)v;
            }
        }
    }

    // ---- local statistics
    const int w = d.w;
    vertical_sums(sm, FW, th, w);
    __syncthreads();
    const unsigned long long n = (unsigned long long)w * (unsigned long long)w;

    if (phase == 1 && two_phase) {
        // sum of D over the tile, exact
        unsigned long long acc = 0;
        for (int oy = warp; oy < th; oy += kThreads / 32) {
            for (int ox = lane; ox < tw; ox += 32) {
                unsigned long long S1 = 0, S2 = 0;
                for (int dx = 0; dx < w; ++dx) {
                    S1 += sm.V1[oy * FW + ox + dx];
                    S2 += sm.V2[oy * FW + ox + dx];
                }
                acc += n * S2 - S1 * S1;
            }
        }
        acc = warp_sum_u64(acc);
        if (lane == 0) bs.red[warp] = acc;
        __threadfence();   // f tile and everything above visible before the done count
        __syncthreads();
        if (tid == 0) {
            unsigned long long s = 0;
            for (int i = 0; i < kThreads / 32; ++i) s += bs.red[i];
            const unsigned long long old = atomicAdd(&d.ctl->sumD_lo, s);
            if (old + s < old) atomicAdd(&d.ctl->sumD_hi, 1ull);
            __threadfence();
            atomicAdd(&d.ctl->p1_done, 1u);
        }
        return;
    }

    // ---- Wiener apply
    double nu2 = d.noise_var;
    if (two_phase) {
        unsigned long long lo, hi;
        lo = __ldcg(&d.ctl->sumD_lo);
        hi = __ldcg(&d.ctl->sumD_hi);
        const double denom = (double)n * (double)n * (double)d.H * (double)d.W;
        nu2 = __ddiv_rn(u128_to_double(hi, lo), denom);
    }
    if (tile == 0 && tid == 0 && d.noise_var_out) *d.noise_var_out = nu2;
    const float v2 = __double2float_rn(nu2);
    const float inv_n = __frcp_rn((float)n);
    const float inv_n2 = __frcp_rn((float)(n * n));
    const float maxv = (float)d.maxv;
    for (int oy = warp; oy < th; oy += kThreads / 32) {
        uint8_t *row = d.dst + (long long)(y0 + oy) * d.dst_pitch;
        for (int ox = lane; ox < tw; ox += 32) {
            unsigned long long S1 = 0, S2 = 0;
            for (int dx = 0; dx < w; ++dx) {
                S1 += sm.V1[oy * FW + ox + dx];
                S2 += sm.V2[oy * FW + ox + dx];
            }
            const unsigned long long D = n * S2 - S1 * S1;
            const unsigned fv = sm.fs[(oy + Rw) * FW + ox + Rw];
            const float mu = __fmul_rn(__ull2float_rn(S1), inv_n);
            const float s2 = __fmul_rn(__ull2float_rn(D), inv_n2);
            const float den = fmaxf(s2, v2);
            const float num = fmaxf(__fsub_rn(s2, v2), 0.0f);
            float y;
            if (den > 0.0f) {
                const float gain = __fdiv_rn(num, den);
                const float dev = __fsub_rn(__uint2float_rn(fv), mu);
                y = __fadd_rn(mu, __fmul_rn(gain, dev));
            } else {
                y = mu;
            }
            float q = floorf(__fadd_rn(y, 0.5f));
            q = fminf(fmaxf(q, 0.0f), maxv);
            const unsigned out = (unsigned)q;
            if (d.elem == 1) row[x0 + ox] = (uint8_t)out;
            else reinterpret_cast<unsigned short *>(row)[x0 + ox] = (unsigned short)out;
            if (d.y_out) d.y_out[(long long)(y0 + oy) * d.W + x0 + ox] = y;
        }
    }
}

__global__ void __launch_bounds__(kThreads) hd_persistent_kernel(const __grid_constant__ LaunchParams lp)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ BlockShared bs;
    const SmemLayout L = layout(lp.tile_w, lp.tile_h, lp.ra_max, lp.rw_max);
    Smem sm;
    sm.V2 = reinterpret_cast<unsigned long long *>(smem_raw + L.v2);
    sm.V1 = reinterpret_cast<unsigned int *>(smem_raw + L.v1);
    sm.wl0 = reinterpret_cast<unsigned int *>(smem_raw + L.wl0);
    sm.wl1 = reinterpret_cast<unsigned int *>(smem_raw + L.wl1);
    sm.gs = reinterpret_cast<unsigned short *>(smem_raw + L.gs);
    sm.fs = reinterpret_cast<unsigned short *>(smem_raw + L.fs);

    const Seg *segs = lp.segs ? lp.segs : lp.oneseg;
    int buf = 0;
    int item;
    if (lp.ticket) {
        if (threadIdx.x == 0) bs.item[0] = (int)atomicAdd(lp.ticket, 1u);
        __syncthreads();
        item = bs.item[0];
    } else {
        item = blockIdx.x;
    }
    while (item < lp.total_items) {
        int lo = 0, hi = lp.nsegs - 1;
        while (lo < hi) {           // last segment with first <= item
            const int mid = (lo + hi + 1) >> 1;
            if (segs[mid].first <= item) lo = mid;
            else hi = mid - 1;
        }
        const Seg sg = segs[lo];
        const ImgDesc &d = lp.descs ? lp.descs[sg.img] : lp.one;
        bool prefetched = false;
        if (lp.ticket && sg.phase == 1) {
            if (threadIdx.x == 0) bs.item[buf ^ 1] = (int)atomicAdd(lp.ticket, 1u);
            prefetched = true;
        }
        run_item(d, sg.phase, item - sg.first, lp, sm, bs, buf ^ 1, prefetched);
        __syncthreads();
        if (lp.ticket) {
            buf ^= 1;
            item = bs.item[buf];
        } else {
            item += gridDim.x;
        }
    }
    // The last CTA out leaves the queue counters and control blocks zeroed
    // for the next launch on this workspace.
    if (lp.ticket && threadIdx.x == 0) {
        __threadfence();
        const unsigned done = atomicAdd(lp.ticket + 1, 1u);
        if (done == gridDim.x - 1) {
            __threadfence();
            for (int i = 0; i < lp.nctl; ++i) {
                lp.ctl_reset[i].sumD_lo = 0;
                lp.ctl_reset[i].sumD_hi = 0;
                lp.ctl_reset[i].p1_done = 0;
            }
            lp.ticket[0] = 0;
            lp.ticket[1] = 0;
            __threadfence();
        }
    }
}

}  // namespace

size_t smem_bytes(int tile_w, int tile_h, int ra_max, int rw_max)
{
    return layout(tile_w, tile_h, ra_max, rw_max).total;
}

int launch_persistent(const LaunchParams &lp, int grid, size_t smem, void *stream)
{
    static size_t configured = 0;
    if (smem > 48 * 1024 && smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(hd_persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return (int)e;
        configured = smem;
    }
    hd_persistent_kernel<<<grid, kThreads, smem, (cudaStream_t)stream>>>(lp);
    return (int)cudaGetLastError();
}

int max_ctas_per_sm(size_t smem)
{
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(hd_persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return 0;
    }
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, hd_persistent_kernel, kThreads, smem) != cudaSuccess)
        return 0;
    return n;
}

int sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return n;
}

int read_and_clear_device_error(unsigned int *out)
{
    unsigned int v = 0, zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_device_error, sizeof(v));
    if (e != cudaSuccess) return (int)e;
    if (v) {
        e = cudaMemcpyToSymbol(g_device_error, &zero, sizeof(zero));
        if (e != cudaSuccess) return (int)e;
    }
    *out = v;
    return 0;
}

}  // namespace hd
