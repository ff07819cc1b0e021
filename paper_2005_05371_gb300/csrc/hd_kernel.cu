// hd_kernel.cu -- the persistent hybrid-denoise kernel for sm_103a.
//
// One launch runs a whole image (or a batch of images) through
//   phase 1: adaptive median (Algorithm 1, step 6) over a 64-column region in
//            shared memory (the output tile plus the Wiener halo), then the
//            exact integer pieces of the image-wide noise variance;
//   phase 2: Wiener apply (Algorithm 1, step 4d) once every phase-1 tile of
//            that image is done.
// Work items (image, phase, tile) are handed out in ticket order by one
// global counter.  An item only waits on items with earlier tickets, so the
// CTA holding the earliest unfinished ticket always makes progress; a CTA may
// therefore take its next ticket before finishing the current item.  Waits
// are bounded: after lp.spin_limit polls the CTA latches DEVERR_TIMEOUT in
// g_device_error and skips the item.  The last CTA to exit zeroes the queue
// counters for the next launch.
//
// Region geometry.  The f region (median output the Wiener stage reads) is
// at most 64 columns x FH rows.  Its first column is Lm = Rw rounded up to
// an even number left of the output tile (Rw = w/2 rows above and columns
// right), so the region starts on an even image column: pixel pairs (2i,
// 2i+1) of the image and of shared memory line up for 32-bit accesses.  The
// output tile is TW = (64 - Lm - Rw) rounded down to even columns by
// FH - 2 Rw rows.  Lane l owns f columns 2l and 2l+1; each warp owns a band
// of rows.  The noisy-input region adds the median halo Ra = Smax/2.
//
// Median, 3x3 stage: two pixels per lane in one 32-bit word (u16x2 SIMD
// min/max, one instruction each).  Each input row is sorted once per column
// triple and reused by three output rows; the median of nine is med3(max of
// row minima, med3 of row medians, min of row maxima).  Level A / level B
// tests use packed differences (zmin <= z <= zmax lane-wise, so the
// subtractions never borrow).  Pixels failing level A join a shared-memory
// worklist that is re-compacted for each larger window k = 5..Smax, one thread
// per pixel.  Level A at k needs only zmin, zmax and how often each occurs
// (the median equals zmin exactly when zmin fills more than half the window);
// pixels whose level B needs the median are compacted again and get it by
// forgetful selection (k = 5, in registers) or by bisection on the value with
// counting passes.
//
// Noise variance (mean local variance, exact):  sum_p D_p with
// D_p = n*S2_p - S1_p^2 equals n * sum_q M(q) f_q^2 - sum_p S1_p^2, where M(q)
// counts the windows (with the border rule) that contain pixel q, separable
// into row and column counts (n for interior pixels).  Phase 1 needs only the
// box sums S1; both sums are exact per image.
//
// Wiener sums: horizontal box sums H1 = sum f, H2 = sum f^2 per row (one
// thread slides along eight columns), then vertical sliding sums per column
// pair.  When n * maxv < 2^17 the variance numerator D < 2^32, so S2 and D
// are computed in wrapping 32-bit arithmetic and are still exact; otherwise
// 64-bit.  The gain and output use binary32 with a fixed order of correctly
// rounded operations (no contraction):
//   mu  = fl(S1) * fl(1/n)            s2 = fl(D) * fl(1/n^2)      v2 = fl(nu2)
//   den = max(s2, v2)                 num = max(s2 - v2, 0)
//   y   = den > 0 ? mu + (num / den) * (fl(f) - mu) : mu
//   out = min(maxv, floor(y + 0.5))
// nu2 = fl64( fl64(sum D) / (n*n*H*W) ) with a correctly rounded 128-bit to
// binary64 conversion, computed by one thread per CTA and image (binary64 is
// slow on this part).
#include <cuda_runtime.h>
#include <climits>
#include <mutex>
#include <type_traits>
#include <cstdint>
#include <cstring>
#include "hd_internal.h"

namespace hd {

__device__ unsigned int g_device_error;

// Optional per-stage cycle counters (build with -DHD_STAGE_PROFILE): thread 0
// of every CTA adds the clock cycles between consecutive stamps to
// g_stage_cycles[stage].  Compiled out otherwise.
#ifdef HD_STAGE_PROFILE
__device__ unsigned long long g_stage_cycles[32];
#define HD_STAMP_INIT() long long hd_t0_ = clock64()
#define HD_STAMP(i)                                                                  \
    do {                                                                             \
        if (threadIdx.x == 0) {                                                      \
            const long long t_ = clock64();                                          \
            atomicAdd(&g_stage_cycles[i], (unsigned long long)(t_ - hd_t0_));        \
            hd_t0_ = t_;                                                             \
        }                                                                            \
    } while (0)
// Per-CTA global timestamps (ns): kernel start, end of the ticket loop, end
// of the phase-2 wait, end; and the number of items the CTA ran.
__device__ unsigned long long g_cta_t[4096][5];
__device__ __forceinline__ unsigned long long hd_gtime()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
#define HD_CTA_T(i)                                                                  \
    do {                                                                             \
        if (threadIdx.x == 0 && blockIdx.x < 4096) g_cta_t[blockIdx.x][i] = hd_gtime(); \
    } while (0)
// Clock cycles of each phase-1 item, by tile index (single images).
__device__ unsigned int g_tile_cyc[1 << 16];
#define HD_CTA_ITEMS(n)                                                              \
    do {                                                                             \
        if (threadIdx.x == 0 && blockIdx.x < 4096) g_cta_t[blockIdx.x][4] = (n);    \
    } while (0)
#else
#define HD_STAMP_INIT() (void)0
#define HD_STAMP(i) (void)0
#define HD_CTA_T(i) (void)0
#define HD_CTA_ITEMS(n) (void)0
#endif

namespace {

typedef unsigned int u32;
typedef unsigned long long u64;
typedef unsigned short u16;

constexpr int FW = 64;          // f-region width
constexpr int FS = 66;          // f-region row stride in u16 (33 words: rows shift banks)
constexpr int HS = 66;          // row stride of the horizontal-sum planes, in elements (even: 64-bit pairs)
constexpr int kWarps = kThreads / 32;
constexpr u32 FULL = 0xffffffffu;

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }
__host__ __device__ inline int g_stride(int ra) { return FW + 2 * ra + 4; }
// One phase-2 stage: the unit's (mu, s2) pairs, then its f bytes as up to two
// row segments widened to 16-byte boundaries.
constexpr int kStagePlane = kUnitPx * 8;
constexpr int kStageBytes = kStagePlane + kUnitPx * 2 + 64;
static_assert(kStageBytes % 16 == 0, "stage alignment");

struct SmemLayout {
    size_t fs, gs, wl, st, h1, h2, total;
};

// fs is live for the whole item; the median view (gs, worklists) and the
// Wiener view (H1, H2) share the rest.
__host__ __device__ inline SmemLayout layout(int FH, int ra_max, int wide)
{
    SmemLayout L;
    L.fs = 0;
    const size_t scratch = align16((size_t)FH * FS * sizeof(u16));
    size_t a = scratch;
    L.gs = a;
    a = align16(a + (size_t)(FH + 2 * ra_max) * g_stride(ra_max) * sizeof(u16));
    L.wl = a;
    a = align16(a + 2 * (size_t)FH * FW * sizeof(u16));
    // growth state per region pixel (windows of 7 and more): zmin | zmax << 16,
    // then the two counts as bytes
    L.st = a;
    if (ra_max >= 3) a = align16(a + (size_t)FH * FW * (sizeof(u32) + sizeof(u16)));
    size_t b = scratch;
    L.h1 = b;
    b = align16(b + (size_t)FH * HS * sizeof(u32));
    L.h2 = b;
    b = align16(b + (size_t)FH * HS * (wide ? sizeof(u64) : sizeof(u32)));
    L.total = a > b ? a : b;
    // plane-mode phase 2 stages its units over the whole area
    if (L.total < (size_t)kStages * kStageBytes) L.total = (size_t)kStages * kStageBytes;
    return L;
}

struct Geo {
    int x0, y0;      // output tile origin (image coordinates)
    int tw, th;      // output tile size (clipped at the image edge)
    int Rw, Ry, Lm, hx;  // Wiener halo (columns right: Rw, rows above/below: Ry), left margin, Lm - Rw
    int Ra, pa;      // median halo, column pad of the g region (Ra + pa is even)
    int GS;          // g-region row stride (u16)
    int ncol, nrow;  // f-region size: Lm + tw + Rw columns, th + 2 Ry rows
    int gfx, gfy;    // image coordinates of f-region cell (0, 0)
};

// Half-sample symmetric extension with period 2n, valid for any i.
__device__ __forceinline__ int refl(int i, int n)
{
    if ((unsigned)i < (unsigned)n) return i;
    const int p = 2 * n;
    int m = i % p;
    if (m < 0) m += p;
    return m < n ? m : p - 1 - m;
}

__device__ __forceinline__ u32 umin(u32 a, u32 b) { return a < b ? a : b; }
__device__ __forceinline__ u32 umax(u32 a, u32 b) { return a > b ? a : b; }
__device__ __forceinline__ u32 vmin(u32 a, u32 b) { return __vminu2(a, b); }
__device__ __forceinline__ u32 vmax(u32 a, u32 b) { return __vmaxu2(a, b); }
__device__ __forceinline__ u32 vmed3(u32 a, u32 b, u32 c) { return vmax(vmin(a, b), vmin(vmax(a, b), c)); }
__device__ __forceinline__ u32 smed3(u32 a, u32 b, u32 c) { return umax(umin(a, b), umin(umax(a, b), c)); }

// ---------------------------------------------------------------- region loads / stores
// cg: through L2 only (data written earlier in this launch by other CTAs);
// otherwise the read-only path.  A runtime flag: one copy of the load code.
template <typename T>
__device__ __forceinline__ T ldg_any(const T *p, bool cg)
{
    return cg ? __ldcg(p) : __ldg(p);
}

// Bytes [lo, hi) of the aligned 16-byte block at blk, by aligned pieces, into
// q0 (bytes 0..7) and q1 (bytes 8..15); nothing outside [lo, hi) is read.
__device__ __noinline__ void load_partial(const uint8_t *blk, int lo, int hi, u64 &q0, u64 &q1, bool cg)
{
    q0 = 0;
    q1 = 0;
    while (lo < hi) {
        u64 v;
        int s;
        if ((lo & 7) == 0 && lo + 8 <= hi) {
            v = ldg_any(reinterpret_cast<const unsigned long long *>(blk + lo), cg);
            s = 8;
        } else if ((lo & 3) == 0 && lo + 4 <= hi) {
            v = ldg_any(reinterpret_cast<const unsigned int *>(blk + lo), cg);
            s = 4;
        } else if ((lo & 1) == 0 && lo + 2 <= hi) {
            v = ldg_any(reinterpret_cast<const unsigned short *>(blk + lo), cg);
            s = 2;
        } else {
            v = ldg_any(blk + lo, cg);
            s = 1;
        }
        if (lo < 8) q0 |= v << (8 * lo);
        else q1 |= v << (8 * (lo - 8));
        lo += s;
    }
}

// Fill a rows x cols shared-memory region (row stride ds u16, first column
// at dst) with the image region whose top-left pixel is (gy0, gx0), gx0 even.
// Rows are read from refl(gy) (or are zero outside, zero_outside); columns
// outside the image are reflected from the loaded columns of the same row (or
// zero).  Global reads are whole aligned 16-byte blocks covering each row's
// bytes; a block may take bytes of a neighbouring row or of the row padding
// (they are not stored) but never leaves the buffer [buf_lo, buf_hi): only
// at the buffer's two ends are aligned narrower pieces used.  Whole blocks
// whose first pixel lands on a 4-byte aligned shared address go to shared
// memory as 32-bit pixel pairs.
__device__ void load_region(u16 *dst, int ds, int rows, int cols, const uint8_t *base, long long pitch, int es,
                            int H, int W, int gy0, int gx0, bool zero_outside, const uint8_t *buf_hi, bool cg)
{
    const int xa = max(gx0, 0), xb = min(gx0 + cols, W);   // in-image columns, xa < xb
    const int J = ((xb - xa) * es + 15) / 16 + 1;          // blocks that can hold a row's bytes
    const int jobs = rows * J;
    constexpr int U = 1;      // one block a pass (more unrolling measured slower: code size)
    for (int j0 = threadIdx.x; j0 < jobs; j0 += kThreads * U) {
        uint4 v[U];
        int lo[U], hi[U], row[U];
        long long xblk[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int job = j0 + u * kThreads;
            lo[u] = 0;
            hi[u] = 0;
            row[u] = 0;
            xblk[u] = 0;
            v[u] = make_uint4(0, 0, 0, 0);
            if (job < jobs) {
                const int r = job / J, bi = job - r * J;
                row[u] = r;
                const int gy = gy0 + r;
                if (zero_outside && (unsigned)gy >= (unsigned)H) continue;
                const uint8_t *rp = base + (long long)refl(gy, H) * pitch;
                const uint8_t *a = rp + (long long)xa * es;
                const uint8_t *b = rp + (long long)xb * es;
                const uint8_t *blk = reinterpret_cast<const uint8_t *>(
                    (reinterpret_cast<uintptr_t>(a) & ~uintptr_t(15)) + 16 * (uintptr_t)bi);
                if (blk >= b) continue;
                lo[u] = blk < a ? (int)(a - blk) : 0;
                hi[u] = blk + 16 > b ? (int)(b - blk) : 16;
                xblk[u] = (long long)(blk - rp);    // byte offset of the block within the row
                if (blk >= base && blk + 16 <= buf_hi) {
                    v[u] = ldg_any(reinterpret_cast<const uint4 *>(blk), cg);
                } else {
                    u64 q0, q1;
                    load_partial(blk, lo[u], hi[u], q0, q1, cg);
                    v[u] = make_uint4((u32)q0, (u32)(q0 >> 32), (u32)q1, (u32)(q1 >> 32));
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (lo[u] >= hi[u]) continue;
            u16 *drow = dst + row[u] * ds;
            const u32 wv[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
            if (es == 1) {
                const int x = (int)xblk[u] - gx0;          // shared column of byte 0
                if ((reinterpret_cast<uintptr_t>(drow + x) & 3) == 0) {
                    u32 *dw = reinterpret_cast<u32 *>(drow + x);
                    if (lo[u] == 0 && hi[u] == 16) {
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            dw[2 * k] = __byte_perm(wv[k], 0u, 0x4140);
                            dw[2 * k + 1] = __byte_perm(wv[k], 0u, 0x4342);
                        }
                    } else {
                        // pairs wholly inside [lo, hi) as 32-bit stores, the ends singly
#pragma unroll
                        for (int k = 0; k < 8; ++k) {
                            const int i0 = 2 * k;
                            const u32 pr = __byte_perm(wv[k >> 1], 0u, (k & 1) ? 0x4342 : 0x4140);
                            if (i0 >= lo[u] && i0 + 1 < hi[u]) dw[k] = pr;
                            else if (i0 >= lo[u] && i0 < hi[u]) drow[x + i0] = (u16)(pr & 0xffffu);
                            else if (i0 + 1 >= lo[u] && i0 + 1 < hi[u]) drow[x + i0 + 1] = (u16)(pr >> 16);
                        }
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (i >= lo[u] && i < hi[u]) drow[x + i] = (u16)((wv[i >> 2] >> (8 * (i & 3))) & 0xffu);
                }
            } else {
                const int x = (int)(xblk[u] >> 1) - gx0;
                if ((reinterpret_cast<uintptr_t>(drow + x) & 3) == 0) {
                    u32 *dw = reinterpret_cast<u32 *>(drow + x);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int i0 = 4 * k;          // byte offset of the pair
                        if (i0 >= lo[u] && i0 + 4 <= hi[u]) dw[k] = wv[k];
                        else if (i0 >= lo[u] && i0 + 2 <= hi[u]) drow[x + 2 * k] = (u16)(wv[k] & 0xffffu);
                        else if (i0 + 2 >= lo[u] && i0 + 4 <= hi[u]) drow[x + 2 * k + 1] = (u16)(wv[k] >> 16);
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 8; ++i)
                        if (2 * i >= lo[u] && 2 * i < hi[u])
                            drow[x + i] = (u16)((wv[i >> 1] >> (16 * (i & 1))) & 0xffffu);
                }
            }
        }
    }
    // halo columns and zero rows
    const bool left = gx0 < 0, right = gx0 + cols > W;
    const bool zrows = zero_outside && (gy0 < 0 || gy0 + rows > H);
    if (left || right || zrows) {
        __syncthreads();
        if (!zero_outside) {
            // reflection: only the halo columns are written
            const int nl = left ? -gx0 : 0, nr = right ? gx0 + cols - W : 0, nh = nl + nr;
            for (int i = threadIdx.x; i < rows * nh; i += kThreads) {
                const int r = i / nh, k = i - r * nh;
                const int c = k < nl ? k : cols - nr + (k - nl);
                const int sc = refl(gx0 + c, W) - gx0;
                dst[r * ds + c] = (sc >= 0 && sc < cols) ? dst[r * ds + sc] : (u16)0;
            }
            return;
        }
        for (int i = threadIdx.x; i < rows * cols; i += kThreads) {
            const int r = i / cols, c = i - r * cols;
            const int gx = gx0 + c, gy = gy0 + r;
            const bool xout = (unsigned)gx >= (unsigned)W;
            if (zero_outside && ((unsigned)gy >= (unsigned)H || xout)) {
                dst[r * ds + c] = 0;
            } else if (xout) {
                const int sc = refl(gx, W) - gx0;
                dst[r * ds + c] = (sc >= 0 && sc < cols) ? dst[r * ds + sc] : (u16)0;
            }
        }
    }
}

// Store rows [0, th) x cols [0, tw) of a shared u16 region (row stride ss,
// first element src, even column) to an image at (y0, x0), x0 even; one
// warp per row, one pixel pair per lane (one 16- or 32-bit store when the
// image address allows).
__device__ void store_region(const u16 *src, int ss, int th, int tw, uint8_t *base, long long pitch, int es, int y0,
                             int x0)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = 2 * lane;
    if (c >= tw) return;
    const bool two = c + 1 < tw;
    for (int r = warp; r < th; r += kWarps) {
        uint8_t *px = base + (long long)(y0 + r) * pitch + (long long)(x0 + c) * es;
        const u32 pr = *reinterpret_cast<const u32 *>(src + r * ss + c);
        if (es == 1) {
            if (two && (reinterpret_cast<uintptr_t>(px) & 1) == 0) {
                *reinterpret_cast<u16 *>(px) = (u16)__byte_perm(pr, 0u, 0x4420);
            } else {
                px[0] = (uint8_t)pr;
                if (two) px[1] = (uint8_t)(pr >> 16);
            }
        } else {
            if (two && (reinterpret_cast<uintptr_t>(px) & 3) == 0) {
                *reinterpret_cast<u32 *>(px) = pr;
            } else {
                reinterpret_cast<u16 *>(px)[0] = (u16)pr;
                if (two) reinterpret_cast<u16 *>(px)[1] = (u16)(pr >> 16);
            }
        }
    }
}

// ---------------------------------------------------------------- median, 3x3
// Append the pixels flagged in this warp to a worklist (row << 6 | col).
__device__ __forceinline__ void wl_append(bool flo, bool fhi, int r, int lane, u16 *wl, int *cnt)
{
    const u32 blo = __ballot_sync(FULL, flo), bhi = __ballot_sync(FULL, fhi);
    if ((blo | bhi) == 0u) return;
    int base = 0;
    if (lane == 0) base = atomicAdd(cnt, __popc(blo) + __popc(bhi));
    base = __shfl_sync(FULL, base, 0);
    const u32 lt = (1u << lane) - 1u;
    if (flo) wl[base + __popc(blo & lt)] = (u16)((r << 6) | (2 * lane));
    if (fhi) wl[base + __popc(blo) + __popc(bhi & lt)] = (u16)((r << 6) | (2 * lane + 1));
}

// 3x3 stage, packed: values < 2^15, two pixels per lane.
__device__ void amf3_packed(const ImgDesc &d, const Geo &g, const u16 *gs, u16 *fs, u16 *wl, int *cnt, int FH)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int RS = (g.nrow + kWarps - 1) / kWarps;     // rows per warp
    const int r0 = warp * RS, r1 = min(r0 + RS, g.nrow);
    if (r0 >= r1) return;
    const bool on_lo = 2 * lane < g.ncol, on_hi = 2 * lane + 1 < g.ncol;
    const bool smax3 = d.smax == 3, keep = d.unresolved != 0;
    const u32 *gw = reinterpret_cast<const u32 *>(gs);
    const int GSw = g.GS >> 1;
    const int wb = ((g.Ra + g.pa) >> 1) + lane;
    u32 *fw = reinterpret_cast<u32 *>(fs);

    auto rowsort = [&](int fr, u32 &lo, u32 &mid, u32 &hi, u32 &ctr) {
        const u32 *row = gw + (fr + g.Ra) * GSw + wb;
        const u32 wm = row[-1], w0 = row[0], wp = row[1];
        u32 a = __byte_perm(wm, w0, 0x5432), b = w0, c = __byte_perm(w0, wp, 0x5432);
        ctr = b;
        const u32 l1 = vmin(a, b), h1 = vmax(a, b);
        lo = vmin(l1, c);
        const u32 t = vmax(l1, c);
        mid = vmin(h1, t);
        hi = vmax(h1, t);
    };
    u32 pl, pm, ph, pc, cl, cm, ch, cc;
    rowsort(r0 - 1, pl, pm, ph, pc);
    rowsort(r0, cl, cm, ch, cc);
#pragma unroll 2
    for (int r = r0; r < r1; ++r) {
        u32 nl, nm, nh, nc;
        rowsort(r + 1, nl, nm, nh, nc);
        const u32 zmin = vmin(vmin(pl, cl), nl), maxlo = vmax(vmax(pl, cl), nl);
        const u32 zmax = vmax(vmax(ph, ch), nh), minhi = vmin(vmin(ph, ch), nh);
        const u32 zmed = vmed3(maxlo, vmed3(pm, cm, nm), minhi);
        const u32 zxy = cc;
        // lane-wise zmin <= zmed, zxy <= zmax: the differences never borrow
        const u32 pa_ = (vmin(zmed - zmin, zmax - zmed) + 0x7fff7fffu) & 0x80008000u;   // level A per lane
        const u32 pb_ = (vmin(zxy - zmin, zmax - zxy) + 0x7fff7fffu) & 0x80008000u;    // level B per lane
        const u32 kb = (pb_ >> 15) * 0xffffu;
        u32 out = (zxy & kb) | (zmed & ~kb);
        bool flo = false, fhi = false;
        if (pa_ != 0x80008000u) {
            const u32 fa = ((~pa_ & 0x80008000u) >> 15) * 0xffffu;    // lanes failing level A
            const u32 alt = (smax3 && keep) ? zxy : zmed;
            out = (out & ~fa) | (alt & fa);
            if (!smax3) {
                flo = on_lo && !(pa_ & 0x8000u);
                fhi = on_hi && !(pa_ & 0x80000000u);
            }
        }
        if (on_lo) fw[r * (FS / 2) + lane] = out;
        if (!smax3) wl_append(flo, fhi, r, lane, wl, cnt);
        pl = cl; pm = cm; ph = ch; pc = cc;
        cl = nl; cm = nm; ch = nh; cc = nc;
    }
}

// 3x3 stage, scalar (full 16-bit range): the same schedule, one pixel at a time.
__device__ void amf3_scalar(const ImgDesc &d, const Geo &g, const u16 *gs, u16 *fs, u16 *wl, int *cnt, int FH)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int RS = (g.nrow + kWarps - 1) / kWarps;     // rows per warp
    const int r0 = warp * RS, r1 = min(r0 + RS, g.nrow);
    if (r0 >= r1) return;
    const bool smax3 = d.smax == 3, keep = d.unresolved != 0;
    const int cbase = g.Ra + g.pa + 2 * lane;
    for (int half = 0; half < 2; ++half) {
        const int col = 2 * lane + half;
        const bool on = col < g.ncol;
        const int gc = cbase + half;
        auto rowsort = [&](int fr, u32 &lo, u32 &mid, u32 &hi, u32 &ctr) {
            const u16 *row = gs + (fr + g.Ra) * g.GS + gc;
            u32 a = row[-1], b = row[0], c = row[1];
            ctr = b;
            const u32 l1 = umin(a, b), h1 = umax(a, b);
            lo = umin(l1, c);
            const u32 t = umax(l1, c);
            mid = umin(h1, t);
            hi = umax(h1, t);
        };
        u32 pl, pm, ph, pc, cl, cm, ch, cc;
        rowsort(r0 - 1, pl, pm, ph, pc);
        rowsort(r0, cl, cm, ch, cc);
        for (int r = r0; r < r1; ++r) {
            u32 nl, nm, nh, nc;
            rowsort(r + 1, nl, nm, nh, nc);
            const u32 zmin = umin(umin(pl, cl), nl), maxlo = umax(umax(pl, cl), nl);
            const u32 zmax = umax(umax(ph, ch), nh), minhi = umin(umin(ph, ch), nh);
            const u32 zmed = smed3(maxlo, smed3(pm, cm, nm), minhi);
            const u32 zxy = cc;
            u32 out;
            bool grow = false;
            if (zmin < zmed && zmed < zmax) out = (zmin < zxy && zxy < zmax) ? zxy : zmed;
            else if (smax3) out = keep ? zxy : zmed;
            else { out = zmed; grow = on; }
            if (on) fs[r * FS + col] = (u16)out;
            if (!smax3) wl_append(half == 0 && grow, half == 1 && grow, r, lane, wl, cnt);
            pl = cl; pm = cm; ph = ch; pc = cc;
            cl = nl; cm = nm; ch = nh; cc = nc;
        }
    }
}

// ---------------------------------------------------------------- median, window growth
__device__ __forceinline__ void cex(u32 &a, u32 &b)
{
    const u32 t = umin(a, b);
    b = umax(a, b);
    a = t;
}

// Forgetful selection: min of a[0..S-1] to a[0], max to a[S-1].
template <int S>
__device__ __forceinline__ void minmax_ends(u32 *a)
{
#pragma unroll
    for (int i = 0; i + 1 < S; i += 2) cex(a[i], a[i + 1]);
#pragma unroll
    for (int i = 2; i < S; i += 2) cex(a[0], a[i]);
#pragma unroll
    for (int i = 1; i < S - 1; i += 2) cex(a[i], a[S - 1]);
}

template <int S>
__device__ __forceinline__ void forget_round(u32 *a, u32 v)
{
    minmax_ends<S>(a);
    a[0] = v;     // drop the min (a[0]) and the max (a[S-1]), insert the next sample
}

// Median of the 5x5 window at ctr by forgetful selection: start with 14
// samples; 11 times discard the min and max of the working set (neither can
// be the median of the rest) and add the next sample; the median of the last
// three is the window median.
__device__ u32 median25(const u16 *ctr, int GS)
{
    u32 a[14];
#pragma unroll
    for (int i = 0; i < 14; ++i) a[i] = ctr[(i / 5 - 2) * GS + (i % 5 - 2)];
#define HD_SAMPLE(i) ((u32)ctr[((i) / 5 - 2) * GS + ((i) % 5 - 2)])
    forget_round<14>(a, HD_SAMPLE(14));
    forget_round<13>(a, HD_SAMPLE(15));
    forget_round<12>(a, HD_SAMPLE(16));
    forget_round<11>(a, HD_SAMPLE(17));
    forget_round<10>(a, HD_SAMPLE(18));
    forget_round<9>(a, HD_SAMPLE(19));
    forget_round<8>(a, HD_SAMPLE(20));
    forget_round<7>(a, HD_SAMPLE(21));
    forget_round<6>(a, HD_SAMPLE(22));
    forget_round<5>(a, HD_SAMPLE(23));
    forget_round<4>(a, HD_SAMPLE(24));
#undef HD_SAMPLE
    return smed3(a[0], a[1], a[2]);
}

// One window size for every pixel on the worklist `cur` (n entries):
//   level A holds iff neither zmin nor zmax fills more than half the window
//   (the median equals zmin exactly when #{v == zmin} > (K*K-1)/2, and zmax
//   likewise);
//   level B with zmin < zxy < zmax keeps zxy; otherwise the pixel needs the
//   median and joins the selection list (stored from the top of `nxt`);
//   pixels failing level A go to `nxt` for the next window, or at Smax take
//   the median (zmin or zmax by the counts) or keep zxy.
// The 5 x 5 window is scanned whole; from 7 x 7 on, only the new ring of
// 4(K-1) samples is read and the extremes and their counts of the previous
// window (kept per pixel in `st_mm` / `st_c`) are updated: a ring holding a
// smaller minimum restarts its count, an equal one adds to it.
template <int K>
__device__ void grow_level(const Geo &g, const u16 *gs, u16 *fs, const u16 *cur, int n, u16 *nxt, int cap,
                           int *cnt_next, int *cnt_sel, bool last, bool keep, u32 *st_mm, u16 *st_c)
{
    constexpr int R = K / 2, M0 = (K * K - 1) / 2;
    const int lane = threadIdx.x & 31;
    for (int e0 = 0; e0 < n; e0 += kThreads) {
        const int e = e0 + threadIdx.x;
        bool to_next = false, to_sel = false;
        u32 ent = 0;
        if (e < n) {
            ent = cur[e];
            const int r = (int)(ent >> 6), c = (int)(ent & 63u);
            const u16 *ctr = gs + (r + g.Ra) * g.GS + (c + g.Ra + g.pa);
            const u32 zxy = ctr[0];
            u32 zmin = 0xffffu, zmax = 0u, cmin = 0, cmax = 0;
            if (K == 5) {
#pragma unroll
                for (int dy = -R; dy <= R; ++dy) {
                    const u16 *row = ctr + dy * g.GS;
#pragma unroll
                    for (int dx = -R; dx <= R; ++dx) {
                        const u32 v = row[dx];
                        zmin = umin(zmin, v);
                        zmax = umax(zmax, v);
                    }
                }
#pragma unroll
                for (int dy = -R; dy <= R; ++dy) {
                    const u16 *row = ctr + dy * g.GS;
#pragma unroll
                    for (int dx = -R; dx <= R; ++dx) {
                        const u32 v = row[dx];
                        cmin += v == zmin;
                        cmax += v == zmax;
                    }
                }
            } else {
                const u16 *top = ctr - R * g.GS, *bot = ctr + R * g.GS;
                u32 rmin = 0xffffu, rmax = 0u;
#pragma unroll 2
                for (int dx = -R; dx <= R; ++dx) {
                    const u32 a = top[dx], b = bot[dx];
                    rmin = umin(rmin, umin(a, b));
                    rmax = umax(rmax, umax(a, b));
                }
#pragma unroll 2
                for (int dy = 1 - R; dy < R; ++dy) {
                    const u32 a = ctr[dy * g.GS - R], b = ctr[dy * g.GS + R];
                    rmin = umin(rmin, umin(a, b));
                    rmax = umax(rmax, umax(a, b));
                }
                const u32 mm = st_mm[ent], cc = st_c[ent];
                const u32 pmin = mm & 0xffffu, pmax = mm >> 16;
                zmin = umin(pmin, rmin);
                zmax = umax(pmax, rmax);
                cmin = zmin == pmin ? (cc & 0xffu) : 0u;
                cmax = zmax == pmax ? (cc >> 8) : 0u;
#pragma unroll 2
                for (int dx = -R; dx <= R; ++dx) {
                    const u32 a = top[dx], b = bot[dx];
                    cmin += (a == zmin) + (b == zmin);
                    cmax += (a == zmax) + (b == zmax);
                }
#pragma unroll 2
                for (int dy = 1 - R; dy < R; ++dy) {
                    const u32 a = ctr[dy * g.GS - R], b = ctr[dy * g.GS + R];
                    cmin += (a == zmin) + (b == zmin);
                    cmax += (a == zmax) + (b == zmax);
                }
            }
            if (cmin <= (u32)M0 && cmax <= (u32)M0) {
                if (zmin < zxy && zxy < zmax) {
                    fs[r * FS + c] = (u16)zxy;
                } else {
                    to_sel = true;
                    if (K > 5) st_mm[ent] = zmin | (zmax << 16);
                }
            } else if (last) {
                fs[r * FS + c] = (u16)(keep ? zxy : (cmin > (u32)M0 ? zmin : zmax));
            } else {
                to_next = true;
                // counts reach at most K*K <= 169 before the last window
                st_mm[ent] = zmin | (zmax << 16);
                st_c[ent] = (u16)(cmin | (cmax << 8));
            }
        }
        const u32 bn = __ballot_sync(FULL, to_next), bs_ = __ballot_sync(FULL, to_sel);
        if (bn | bs_) {
            int pn = 0, ps = 0;
            if (lane == 0) {
                if (bn) pn = atomicAdd(cnt_next, __popc(bn));
                if (bs_) ps = atomicAdd(cnt_sel, __popc(bs_));
            }
            pn = __shfl_sync(FULL, pn, 0);
            ps = __shfl_sync(FULL, ps, 0);
            const u32 lt = (1u << lane) - 1u;
            if (to_next) nxt[pn + __popc(bn & lt)] = (u16)ent;
            if (to_sel) nxt[cap - 1 - (ps + __popc(bs_ & lt))] = (u16)ent;
        }
    }
}

// Medians of the K x K windows of the nsel pixels on the selection list
// (stored downward from sel_top).  K = 5: forgetful selection, one thread per
// pixel.  K >= 7: G lanes per pixel (G a power of two, more when the list is
// short) split the window rows; each pass counts c = #{v <= t} at the bracket
// midpoint t and also finds max{v <= t} and min{v > t}, so the bracket
// [lo, hi] (lo <= median <= hi, starting inside (zmin, zmax)) moves onto
// sample values: c > (K*K-1)/2 puts the median at or below max{v <= t},
// otherwise at or above min{v > t}.  Ends when lo == hi: the exact median.
template <int K>
__device__ void select_level(const Geo &g, const u16 *gs, u16 *fs, const u16 *sel_top, int nsel, const u32 *st_mm,
                             int lanes_cap)
{
    constexpr int R = K / 2, M0 = (K * K - 1) / 2;
    if (K == 5) {
        for (int e = threadIdx.x; e < nsel; e += kThreads) {
            const u32 ent = *(sel_top - e);
            const int r = (int)(ent >> 6), c = (int)(ent & 63u);
            fs[r * FS + c] = (u16)median25(gs + (r + g.Ra) * g.GS + (c + g.Ra + g.pa), g.GS);
        }
        return;
    }
    const int GMAX = lanes_cap ? lanes_cap : (K >= 9 ? 8 : 4);
    int G = 1;
    while (G < GMAX && nsel * G * 2 <= kThreads) G *= 2;
    const int gid = threadIdx.x / G, gl = threadIdx.x & (G - 1), ngroups = kThreads / G;
    const int rounds = (nsel + ngroups - 1) / ngroups;
    for (int rd = 0; rd < rounds; ++rd) {
        const int e = rd * ngroups + gid;
        const bool valid = e < nsel;
        u32 ent = 0, lo = 1, hi = 0;
        const u16 *ctr = gs;
        if (valid) {
            ent = *(sel_top - e);
            const int r = (int)(ent >> 6), c = (int)(ent & 63u);
            ctr = gs + (r + g.Ra) * g.GS + (c + g.Ra + g.pa);
            const u32 mm = st_mm[ent];
            lo = (mm & 0xffffu) + 1u;
            hi = (mm >> 16) - 1u;
        }
        // every lane of the warp runs the same number of passes (shuffles)
        while (__any_sync(FULL, lo < hi)) {
            const bool act = lo < hi;
            const u32 t = (lo + hi) >> 1;
            u32 cnt = 0, below = 0, above = 0xffffu;
            if (act) {
#pragma unroll 1
                for (int dy = gl - R; dy <= R; dy += G) {
                    const u16 *row = ctr + dy * g.GS;
#pragma unroll
                    for (int dx = -R; dx <= R; ++dx) {
                        const u32 v = row[dx];
                        const bool le = v <= t;
                        cnt += le;
                        below = umax(below, le ? v : 0u);
                        above = umin(above, le ? 0xffffu : v);
                    }
                }
            }
            for (int m = 1; m < G; m <<= 1) {
                cnt += __shfl_xor_sync(FULL, cnt, m);
                below = umax(below, __shfl_xor_sync(FULL, below, m));
                above = umin(above, __shfl_xor_sync(FULL, above, m));
            }
            if (act) {
                if (cnt > (u32)M0) hi = below;
                else lo = above;
            }
        }
        if (valid && gl == 0) {
            const int r = (int)(ent >> 6), c = (int)(ent & 63u);
            fs[r * FS + c] = (u16)lo;
        }
    }
}

// Medians of the K x K windows (K >= 7) of the nsel pixels on the selection
// list, for values below 2^15.  G lanes per pixel (4 at 7x7, 8 from 9x9)
// split the window's rows and keep their samples in registers, two to a
// 32-bit word (a row's odd last sample, and rows past the window, are padded
// with 0x7fff, which no threshold reaches).  Then bisection on the value:
// the median is the smallest t with c(t) = #{v <= t} > (K*K-1)/2, so c(t) >
// (K*K-1)/2 puts it at or below t, otherwise above.  The bracket starts
// strictly inside (zmin, zmax) (level A holds) and halves every pass:
// ceil(log2(zmax - zmin - 1)) passes.  One word counts both of its samples:
// with both halves below 2^15, ((0x8000 | t) * 0x10001) - w has bit 15 (31)
// set exactly where its low (high) sample is <= t, and no borrow crosses
// from one half into the other.
template <int K>
__device__ void select_level_packed(const Geo &g, const u16 *gs, u16 *fs, const u16 *sel_top, int nsel,
                                    const u32 *st_mm)
{
    constexpr int R = K / 2, M0 = (K * K - 1) / 2;
    constexpr int G = K >= 9 ? 8 : 4;
    constexpr int ROWS = (K + G - 1) / G;      // rows per lane
    constexpr int WPR = (K + 1) / 2;           // words per row
    const int gid = threadIdx.x / G, gl = threadIdx.x & (G - 1);
    constexpr int ngroups = kThreads / G;
    const int rounds = (nsel + ngroups - 1) / ngroups;
    for (int rd = 0; rd < rounds; ++rd) {
        const int e = rd * ngroups + gid;
        u32 ent = 0, lo = 1, hi = 0;
        u32 w[ROWS * WPR];
#pragma unroll
        for (int i = 0; i < ROWS * WPR; ++i) w[i] = 0x7fff7fffu;
        if (e < nsel) {
            ent = *(sel_top - e);
            const int r = (int)(ent >> 6), c = (int)(ent & 63u);
            const u16 *ctr = gs + (r + g.Ra) * g.GS + (c + g.Ra + g.pa);
            const u32 mm = st_mm[ent];
            lo = (mm & 0xffffu) + 1u;
            hi = (mm >> 16) - 1u;
#pragma unroll
            for (int j = 0; j < ROWS; ++j) {
                const int dy = gl - R + j * G;
                const u16 *row = ctr + dy * g.GS;
#pragma unroll
                for (int q = 0; q < WPR; ++q) {
                    const int dx = 2 * q - R;
                    u32 a = 0x7fffu, b = 0x7fffu;
                    if (dy <= R) {
                        a = row[dx];
                        if (dx + 1 <= R) b = row[dx + 1];
                    }
                    w[j * WPR + q] = a | (b << 16);
                }
            }
        }
        // every lane of the warp runs the same number of passes (shuffles)
        while (__any_sync(FULL, lo < hi)) {
            const u32 t = (lo + hi) >> 1;
            const u32 T = (0x8000u | t) * 0x10001u;
            u32 cnt = 0;
#pragma unroll
            for (int i = 0; i < ROWS * WPR; ++i) cnt += ((T - w[i]) >> 15) & 0x10001u;
            cnt = (cnt & 0xffffu) + (cnt >> 16);
#pragma unroll
            for (int m = 1; m < G; m <<= 1) cnt += __shfl_xor_sync(FULL, cnt, m);
            if (lo < hi) {
                if (cnt > (u32)M0) hi = t;
                else lo = t + 1;
            }
        }
        if (e < nsel && gl == 0) {
            const int r = (int)(ent >> 6), c = (int)(ent & 63u);
            fs[r * FS + c] = (u16)lo;
        }
    }
}

// The exact median of the K x K window at ctr, known to lie strictly between
// zmin and zmax, by one thread: the same value-snapping bisection as the
// cooperative selection, over the whole window.
template <int K>
__device__ u32 median_snap(const u16 *ctr, int GS, u32 zmin, u32 zmax)
{
    constexpr int R = K / 2, M0 = (K * K - 1) / 2;
    u32 lo = zmin + 1, hi = zmax - 1;
    while (lo < hi) {
        const u32 t = (lo + hi) >> 1;
        u32 c = 0, below = 0, above = 0xffffu;
#pragma unroll 1
        for (int dy = -R; dy <= R; ++dy) {
            const u16 *row = ctr + dy * GS;
#pragma unroll
            for (int dx = -R; dx <= R; ++dx) {
                const u32 v = row[dx];
                const bool le = v <= t;
                c += le;
                below = umax(below, le ? v : 0u);
                above = umin(above, le ? 0xffffu : v);
            }
        }
        if (c > (u32)M0) hi = below;
        else lo = above;
    }
    return lo;
}

// Levels A and B of one pixel for the K x K window (whole-window extremes and
// counts); returns true with the output in `out` when the pixel is resolved.
template <int K>
__device__ __forceinline__ bool level_one(const u16 *ctr, int GS, u32 zxy, bool last, bool keep, u32 &out)
{
    constexpr int R = K / 2, M0 = (K * K - 1) / 2;
    u32 zmin = 0xffffu, zmax = 0u, cmin = 0, cmax = 0;
#pragma unroll 1
    for (int dy = -R; dy <= R; ++dy) {
        const u16 *row = ctr + dy * GS;
#pragma unroll
        for (int dx = -R; dx <= R; ++dx) {
            const u32 v = row[dx];
            zmin = umin(zmin, v);
            zmax = umax(zmax, v);
        }
    }
#pragma unroll 1
    for (int dy = -R; dy <= R; ++dy) {
        const u16 *row = ctr + dy * GS;
#pragma unroll
        for (int dx = -R; dx <= R; ++dx) {
            const u32 v = row[dx];
            cmin += v == zmin;
            cmax += v == zmax;
        }
    }
    if (cmin <= (u32)M0 && cmax <= (u32)M0) {
        if (zmin < zxy && zxy < zmax) out = zxy;
        else out = K == 5 ? median25(ctr, GS) : median_snap<K>(ctr, GS, zmin, zmax);
        return true;
    }
    if (last) {
        out = keep ? zxy : (cmin > (u32)M0 ? zmin : zmax);
        return true;
    }
    return false;
}

// Warp 0, when at most 32 pixels failed level A at 3x3: one pixel per lane
// through the windows k = 5..Smax, with no block barriers (the worklist path
// pays two or three per window size for a handful of pixels).
__device__ void grow_small(const ImgDesc &d, const Geo &g, const u16 *gs, u16 *fs, const u16 *list, int n)
{
    const int lane = threadIdx.x & 31;
    if (lane >= n) return;
    const u32 ent = list[lane];
    const int r = (int)(ent >> 6), c = (int)(ent & 63u);
    const u16 *ctr = gs + (r + g.Ra) * g.GS + (c + g.Ra + g.pa);
    const u32 zxy = ctr[0];
    const bool keep = d.unresolved != 0;
    u32 out = zxy;
    for (int k = 5; k <= d.smax; k += 2) {
        const bool last = k == d.smax;
        bool done;
        switch (k) {
        case 5: done = level_one<5>(ctr, g.GS, zxy, last, keep, out); break;
        case 7: done = level_one<7>(ctr, g.GS, zxy, last, keep, out); break;
        case 9: done = level_one<9>(ctr, g.GS, zxy, last, keep, out); break;
        case 11: done = level_one<11>(ctr, g.GS, zxy, last, keep, out); break;
        case 13: done = level_one<13>(ctr, g.GS, zxy, last, keep, out); break;
        default: done = level_one<15>(ctr, g.GS, zxy, last, keep, out); break;
        }
        if (done) break;
    }
    fs[r * FS + c] = (u16)out;
}

// Windows k = 5..Smax for the pixels that failed level A at k = 3.
template <bool PACK>
__device__ void amf_grow(const ImgDesc &d, const Geo &g, const u16 *gs, u16 *fs, u16 *wl0, u16 *wl1, int *cnt,
                         int cap, u32 *st_mm, u16 *st_c, int small_growth, int lanes_cap)
{
    const int n0 = cnt[0];
    HD_STAMP_INIT();
    if (n0 <= small_growth) {
        if (n0 > 0 && threadIdx.x < 32) grow_small(d, g, gs, fs, wl0, n0);
        HD_STAMP(11);
        return;
    }
    const bool keep = d.unresolved != 0;
    u16 *cur = wl0, *nxt = wl1;
    int ci = 0;
    for (int k = 5; k <= d.smax; k += 2) {
        const int n = cnt[ci];
        if (n == 0) break;
        if (threadIdx.x == 0) {
            cnt[ci ^ 1] = 0;
            cnt[2] = 0;
        }
        __syncthreads();
        const bool last = k == d.smax;
        switch (k) {
        case 5: grow_level<5>(g, gs, fs, cur, n, nxt, cap, &cnt[ci ^ 1], &cnt[2], last, keep, st_mm, st_c); break;
        case 7: grow_level<7>(g, gs, fs, cur, n, nxt, cap, &cnt[ci ^ 1], &cnt[2], last, keep, st_mm, st_c); break;
        case 9: grow_level<9>(g, gs, fs, cur, n, nxt, cap, &cnt[ci ^ 1], &cnt[2], last, keep, st_mm, st_c); break;
        case 11: grow_level<11>(g, gs, fs, cur, n, nxt, cap, &cnt[ci ^ 1], &cnt[2], last, keep, st_mm, st_c); break;
        case 13: grow_level<13>(g, gs, fs, cur, n, nxt, cap, &cnt[ci ^ 1], &cnt[2], last, keep, st_mm, st_c); break;
        default: grow_level<15>(g, gs, fs, cur, n, nxt, cap, &cnt[ci ^ 1], &cnt[2], last, keep, st_mm, st_c);
            break;
        }
        __syncthreads();
        HD_STAMP(8);
        const int nsel = cnt[2];
        if (nsel > 0) {
            const u16 *top = nxt + cap - 1;
            if (PACK) {
                switch (k) {
                case 5: select_level<5>(g, gs, fs, top, nsel, st_mm, lanes_cap); break;
                case 7: select_level_packed<7>(g, gs, fs, top, nsel, st_mm); break;
                case 9: select_level_packed<9>(g, gs, fs, top, nsel, st_mm); break;
                case 11: select_level_packed<11>(g, gs, fs, top, nsel, st_mm); break;
                case 13: select_level_packed<13>(g, gs, fs, top, nsel, st_mm); break;
                default: select_level_packed<15>(g, gs, fs, top, nsel, st_mm); break;
                }
            } else {
                switch (k) {
                case 5: select_level<5>(g, gs, fs, top, nsel, st_mm, lanes_cap); break;
                case 7: select_level<7>(g, gs, fs, top, nsel, st_mm, lanes_cap); break;
                case 9: select_level<9>(g, gs, fs, top, nsel, st_mm, lanes_cap); break;
                case 11: select_level<11>(g, gs, fs, top, nsel, st_mm, lanes_cap); break;
                case 13: select_level<13>(g, gs, fs, top, nsel, st_mm, lanes_cap); break;
                default: select_level<15>(g, gs, fs, top, nsel, st_mm, lanes_cap); break;
                }
            }
            __syncthreads();
            HD_STAMP(k == 5 ? 9 : 10);
        }
        u16 *t = cur; cur = nxt; nxt = t;
        ci ^= 1;
    }
}

// ---------------------------------------------------------------- Wiener sums
// Horizontal box sums of f over the w-column window of every output column
// x in [0, tw), for f rows [0, nrow):
//   H1[j][x] = sum_{t<w} f[j][x + hx + t],  H2 = the same of f^2.
// One thread slides along eight columns of one row; the lanes of a warp take
// 32 consecutive rows (conflict-free shared reads).  NARROW: H2 as u32
// (exact values; the S2 sums built from them may wrap), WIDE: H2 as u64.
template <bool NARROW>
__device__ void hsums(const Geo &g, const u16 *fs, u32 *H1, void *h2p, int w, bool with_h2)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int groups = (g.nrow + 31) >> 5, runs = (g.tw + 7) >> 3;
    for (int job = warp; job < groups * runs; job += kWarps) {
        const int grp = job / runs, m = job - grp * runs;
        const int j = grp * 32 + lane;
        if (j >= g.nrow) continue;
        const int xs = 8 * m, xe = min(xs + 8, g.tw);
        const u16 *fr = fs + j * FS + g.hx;
        u32 *h1 = H1 + j * HS;
        // NARROW: the window sums of f^2 are exact in 32 bits
        using S2 = typename std::conditional<NARROW, u32, u64>::type;
        u32 s1 = 0;
        S2 s2 = 0;
        for (int t = 0; t < w; ++t) {
            const u32 f = fr[xs + t];
            s1 += f;
            if (with_h2) s2 += (S2)(f * f);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int x = xs + i;
            if (x < xe) {
                h1[x] = s1;
                if (with_h2) {
                    if (NARROW) reinterpret_cast<u32 *>(h2p)[j * HS + x] = (u32)s2;
                    else reinterpret_cast<u64 *>(h2p)[j * HS + x] = (u64)s2;
                }
                if (x + 1 < xe) {
                    const u32 a = fr[x + w], b = fr[x];
                    s1 += a - b;
                    if (with_h2) {
                        s2 += (S2)(a * a);
                        s2 -= (S2)(b * b);
                    }
                }
            }
        }
    }
}

// Number of (pixel, window offset) pairs whose sample lands on index y of an
// axis of length N under the border rule (window radius r).
__device__ u32 window_multiplicity(int y, int N, int r, bool zero)
{
    if (zero) return (u32)(min(r, y) + min(r, N - 1 - y) + 1);
    if (y >= r && y <= N - 1 - r) return (u32)(2 * r + 1);
    u32 m = 0;
    const long long lo = -r, hi = (long long)N - 1 + r, P = 2LL * N;
    for (int fam = 0; fam < 2; ++fam) {
        const long long base = fam ? (-1LL - y) : (long long)y;     // refl(t) == y
        long long k = (lo - base) >= 0 ? (lo - base + P - 1) / P : -((base - lo) / P);
        for (long long t = base + k * P; t <= hi; t += P) {
            if (t < lo) continue;
            const long long a = max(-(long long)r, t - N + 1), b = min((long long)r, t);
            if (b >= a) m += (u32)(b - a + 1);
        }
    }
    return m;
}

// ---------------------------------------------------------------- exactness helpers
__device__ __forceinline__ u64 warp_sum_u64(u64 x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(FULL, x, o);
    return x;
}

// Add v to the split sum (lo32 + hi32 * 2^32): two fire-and-forget reductions.
__device__ __forceinline__ void split_add(u64 *lo32, u64 *hi32, u64 v)
{
    atomicAdd(lo32, v & 0xffffffffull);
    atomicAdd(hi32, v >> 32);
}

// hi32 * 2^32 + lo32 as a 128-bit value {hi, lo}.
__device__ __forceinline__ void split_total(u64 lo32, u64 hi32, u64 &hi, u64 &lo)
{
    lo = lo32 + (hi32 << 32);
    hi = (hi32 >> 32) + (lo < lo32 ? 1ull : 0ull);
}

// Correctly rounded conversion of hi*2^64 + lo to binary64.
__device__ double u128_to_double(u64 hi, u64 lo)
{
    if (hi == 0) return __ull2double_rn(lo);
    const int s = __clzll((long long)hi);
    u64 top = s == 0 ? hi : ((hi << s) | (lo >> (64 - s)));
    const u64 rest = lo << s;
    top |= (rest != 0ull) ? 1ull : 0ull;    // sticky bit, far below the rounding position
    // exact scaling by 2^(64 - s) (1 <= 64 - s <= 64: a normal power of two)
    return __ull2double_rn(top) * __longlong_as_double((long long)(1023 + 64 - s) << 52);
}

// nu2 = fl(fl(n * B - A) / (n^2 H W)) from the two exact per-image sums.  The
// quotient a / b uses the reciprocal y = RN(1 / b) from the host and
// Markstein's correction (P. Markstein, IBM J. Res. Dev. 34(1), 1990): with
// q0 = RN(a y) (within an ulp of a / b) and the exact remainder r = a - b q0
// (one fused multiply-add), RN(q0 + r y) = RN(a / b).  b = n^2 H W < 2^53 is
// exact; a is far from overflow and underflow.
__device__ double noise_variance(const ImgCtl *ctl, u64 n, int H, int W, double inv_den)
{
    u64 alo, ahi, blo, bhi;
    split_total(__ldcg(&ctl->A_lo32), __ldcg(&ctl->A_hi32), ahi, alo);
    split_total(__ldcg(&ctl->B_lo32), __ldcg(&ctl->B_hi32), bhi, blo);
    const u64 nlo = blo * n;
    const u64 nhi = __umul64hi(blo, n) + bhi * n;
    const u64 dlo = nlo - alo;
    const u64 dhi = nhi - ahi - (nlo < alo ? 1ull : 0ull);
    const double denom = (double)n * (double)n * (double)H * (double)W;
    const double a = u128_to_double(dhi, dlo);
    const double q0 = __dmul_rn(a, inv_den);
    const double r = __fma_rn(-denom, q0, a);
    return __fma_rn(r, inv_den, q0);
}

__device__ bool wait_phase1(const ImgDesc &d, u32 total, u64 limit, int *s_flag)
{
    if (threadIdx.x == 0) {
        int ok = 1;
        u64 polls = 0;
        volatile u32 *cnt = &d.ctl->p1_done;
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

struct P2Stage {
    u32 p0;           // first pixel of the unit (row-major index)
    int n;            // its pixels (at most kUnitPx; 0: the stage is empty)
    int y0, x0;       // row and column of p0
    int na;           // pixels of the unit in row y0
    int fa, fb;       // stage offsets of f for row y0 and row y0 + 1 (-1: f not staged)
};

struct BlockShared {
    int item[2];      // current / next ticket (double buffer)
    Seg seg[2];       //   its segment
    ImgDesc desc[2];  //   its image's descriptor (batches; single images read the launch parameters)
    u64 full[kStages];        // plane-mode phase 2: stage s staged (bulk-copy bytes landed)
    P2Stage st[kStages];      //   what each stage holds
    u32 fullpar;              //   bit s: parity of the next phase to wait for on stage s
    const ImgCtl *nu2_of;   // image whose noise variance is cached below
    double nu2;
    float nu2f;
    int cnt[3];
    int flag;
    u64 red[2][kWarps];
    u32 my[128];
    u32 mx[FW];
};

// ---------------------------------------------------------------- Wiener passes
struct ApplyConst {
    u32 n;
    float v2f, inv_n, inv_n2;
    u32 maxv;
};

// Phase-1 statistics of one tile: sum over its pixels of S1^2 (A) and of
// M(q) f_q^2 (B), added to the image's exact sums.  With a plane, the tile's
// binary32 mu = fl(S1)*fl(1/n) and s2 = fl(D)*fl(1/n^2) (neither depends on the
// noise variance) are stored for phase 2, which then needs no sums and no halo.
template <bool NARROW, bool PLANE>
__device__ void tile_stats(const ImgDesc &d, const Geo &g, const u16 *fs, u32 *H1, void *h2p, BlockShared &bs)
{
    const int w = d.w, wy = d.wh;      // window columns, rows
    constexpr bool with_plane = PLANE;
    HD_STAMP_INIT();
    // H1 (and H2 with a plane) are in place: run_item_t ran hsums
    const bool zero = d.border_zero != 0;
    const int gy0 = g.y0 + d.gy_off;       // the tile's first row in the whole image
    const bool interior = !zero && gy0 >= g.Ry && gy0 + g.th <= d.Hg - g.Ry && g.x0 >= g.Rw &&
                          g.x0 + g.tw <= d.W - g.Rw;
    if (!interior) {
        for (int i = threadIdx.x; i < g.th + g.tw; i += kThreads) {
            if (i < g.th) bs.my[i] = window_multiplicity(gy0 + i, d.Hg, g.Ry, zero);
            else bs.mx[i - g.th] = window_multiplicity(g.x0 + i - g.th, d.W, g.Rw, zero);
        }
    }
    __syncthreads();
    HD_STAMP(16);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x = 2 * lane;
    const int per = (g.th + kWarps - 1) / kWarps;
    const int j0 = warp * per, j1 = min(j0 + per, g.th);
    u64 accA = 0, accB = 0;
    if (x < g.tw && j0 < j1) {
        const bool two = x + 1 < g.tw;
        const u32 n = (u32)(w * wy);
        const float inv_n = __frcp_rn((float)n), inv_n2 = __frcp_rn((float)(n * n));
        const u32 *H2n = reinterpret_cast<const u32 *>(h2p);
        const u64 *H2w = reinterpret_cast<const u64 *>(h2p);
        u32 sa = 0, sb = 0, qa = 0, qb = 0;
        u64 wa = 0, wb = 0;
        for (int t = 0; t < wy; ++t) {
            const uint2 h = *reinterpret_cast<const uint2 *>(H1 + (j0 + t) * HS + x);
            sa += h.x;
            sb += h.y;
            if (with_plane) {
                if (NARROW) {
                    const uint2 q = *reinterpret_cast<const uint2 *>(H2n + (j0 + t) * HS + x);
                    qa += q.x;
                    qb += q.y;
                } else {
                    wa += H2w[(j0 + t) * HS + x];
                    wb += H2w[(j0 + t) * HS + x + 1];
                }
            }
        }
        float2 *pp = with_plane ? reinterpret_cast<float2 *>(d.plane) + (long long)(g.y0 + j0) * d.W + g.x0 + x
                                : nullptr;
        const bool pair16 = two && ((d.W | g.x0) & 1) == 0 &&
                            (reinterpret_cast<uintptr_t>(d.plane) & 15) == 0;   // (mu, s2) pairs land 16-byte aligned
        for (int j = j0; j < j1; ++j) {
            const u32 fp = *reinterpret_cast<const u32 *>(fs + (j + g.Ry) * FS + g.Lm + x);
            const u32 fa = fp & 0xffffu, fb = fp >> 16;
            if (interior) {
                accA += (u64)sa * sa + (two ? (u64)sb * sb : 0ull);
                accB += (u64)(fa * fa) + (two ? (u64)(fb * fb) : 0ull);
            } else {
                const u32 my = bs.my[j];
                accA += (u64)sa * sa;
                accB += (u64)(fa * fa) * (my * bs.mx[x]);
                if (two) {
                    accA += (u64)sb * sb;
                    accB += (u64)(fb * fb) * (my * bs.mx[x + 1]);
                }
            }
            if (with_plane) {
                float da, db;
                if (NARROW) {
                    da = __uint2float_rn(n * qa - sa * sa);     // exact: the true value is < 2^32
                    db = __uint2float_rn(n * qb - sb * sb);
                } else {
                    da = __ull2float_rn((u64)n * wa - (u64)sa * sa);
                    db = __ull2float_rn((u64)n * wb - (u64)sb * sb);
                }
                const float mua = __fmul_rn(__uint2float_rn(sa), inv_n), s2a = __fmul_rn(da, inv_n2);
                const float mub = __fmul_rn(__uint2float_rn(sb), inv_n), s2b = __fmul_rn(db, inv_n2);
                if (pair16 || (two && (reinterpret_cast<uintptr_t>(pp) & 15) == 0)) {
                    *reinterpret_cast<float4 *>(pp) = make_float4(mua, s2a, mub, s2b);
                } else {
                    pp[0] = make_float2(mua, s2a);
                    if (two) pp[1] = make_float2(mub, s2b);
                }
                pp += d.W;
            }
            if (j + 1 < j1) {
                const uint2 hi_ = *reinterpret_cast<const uint2 *>(H1 + (j + wy) * HS + x);
                const uint2 ho_ = *reinterpret_cast<const uint2 *>(H1 + j * HS + x);
                sa += hi_.x - ho_.x;
                sb += hi_.y - ho_.y;
                if (with_plane) {
                    if (NARROW) {
                        const uint2 qi = *reinterpret_cast<const uint2 *>(H2n + (j + wy) * HS + x);
                        const uint2 qo = *reinterpret_cast<const uint2 *>(H2n + j * HS + x);
                        qa += qi.x - qo.x;
                        qb += qi.y - qo.y;
                    } else {
                        wa += H2w[(j + wy) * HS + x];
                        wa -= H2w[j * HS + x];
                        wb += H2w[(j + wy) * HS + x + 1];
                        wb -= H2w[j * HS + x + 1];
                    }
                }
            }
        }
    }
    HD_STAMP(17);
    if (interior) accB *= (u64)w * (u64)wy;
    accA = warp_sum_u64(accA);
    accB = warp_sum_u64(accB);
    if (lane == 0) {
        bs.red[0][warp] = accA;
        bs.red[1][warp] = accB;
    }
    __syncthreads();
    HD_STAMP(18);
    if (threadIdx.x == 0) {
        u64 sa = 0, sb = 0;
        for (int i = 0; i < kWarps; ++i) {
            sa += bs.red[0][i];
            sb += bs.red[1][i];
        }
        split_add(&d.ctl->A_lo32, &d.ctl->A_hi32, sa);
        split_add(&d.ctl->B_lo32, &d.ctl->B_hi32, sb);
        // release: the CTA's f tile and plane (ordered before this thread by
        // the barrier) and the sums become visible before the done count
        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&d.ctl->p1_done) : "memory");
    }
}

// binary32 Wiener output of one pixel (fixed evaluation order, see top).
__device__ __forceinline__ u32 wiener_px(u32 s1, float dfl, u32 fv, const ApplyConst &k, float &y)
{
    const float mu = __fmul_rn(__uint2float_rn(s1), k.inv_n);
    const float s2 = __fmul_rn(dfl, k.inv_n2);
    const float den = fmaxf(s2, k.v2f);
    const float num = fmaxf(__fsub_rn(s2, k.v2f), 0.0f);
    // num = 0 (local variance at or below the noise level: most pixels of flat
    // areas, and every pixel with den = 0) gives gain = +0 and y = mu + (+-0)
    // = mu exactly (mu >= +0); only num > 0 (then den >= num) needs the divide
    if (num > 0.0f) {
        const float gain = __fdiv_rn(num, den);
        y = __fadd_rn(mu, __fmul_rn(gain, __fsub_rn(__uint2float_rn(fv), mu)));
    } else {
        y = mu;
    }
    // floor(y + 0.5) clamped to [0, maxv]: the round-down conversion saturates
    // negatives (and NaN) to 0
    return min(__float2uint_rd(__fadd_rn(y, 0.5f)), k.maxv);
}

// binary32 Wiener output from the stored (mu, s2) of a pixel.
__device__ __forceinline__ u32 wiener_ms(float mu, float s2, u32 fv, const ApplyConst &k, float &y)
{
    const float den = fmaxf(s2, k.v2f);
    const float num = fmaxf(__fsub_rn(s2, k.v2f), 0.0f);
    // num = 0 (local variance at or below the noise level: most pixels of flat
    // areas, and every pixel with den = 0) gives gain = +0 and y = mu + (+-0)
    // = mu exactly (mu >= +0); only num > 0 (then den >= num) needs the divide
    if (num > 0.0f) {
        const float gain = __fdiv_rn(num, den);
        y = __fadd_rn(mu, __fmul_rn(gain, __fsub_rn(__uint2float_rn(fv), mu)));
    } else {
        y = mu;
    }
    // floor(y + 0.5) clamped to [0, maxv]: the round-down conversion saturates
    // negatives (and NaN) to 0
    return min(__float2uint_rd(__fadd_rn(y, 0.5f)), k.maxv);
}

// ---------------------------------------------------------------- plane-mode phase 2
// Every CTA applies its own contiguous share of the image's pixels (all CTAs
// reach phase 2 together, at the image-wide barrier, so equal shares are
// balanced).  Two ways, chosen on the host by the working set: straight from
// L2 (p2_direct, below), or in units of up to kUnitPx pixels staged in shared
// memory by bulk copies (cp.async.bulk, completion counted on an mbarrier per
// stage) up to kStages units ahead of the one being applied (p2_share).
// There thread 0 issues the copies; all threads apply; a block barrier per
// unit frees its stage for the next copy.
__device__ __forceinline__ u32 smem_addr(const void *p) { return (u32)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(u64 *m, u32 count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(m)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(u64 *m, u32 bytes)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(m)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(u64 *m, u32 parity)
{
    u32 ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_addr(m)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Bounded wait for the completion of phase `parity` of an mbarrier.
__device__ bool mbar_wait(u64 *m, u32 parity, u64 limit)
{
    for (u64 i = 0;; ++i) {
        if (mbar_try_wait(m, parity)) return true;
        if (i >= limit) return false;
        if (i >= 64) __nanosleep(256);
    }
}

__device__ __forceinline__ void bulk_copy(void *dst, const void *src, u32 bytes, u64 *m)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(m))
                 : "memory");
}

// Thread 0: stage pixels [q0, q0 + n) of image d into stage s; q0 - own0 W is
// even and the plane base puts that pixel's pair on a 16-byte boundary.
// Every address and size is a multiple of 16 bytes and stays inside its
// buffer: the plane is allocated in whole 256-byte blocks with 16 bytes to
// spare, f rows have a 16-byte-multiple pitch.
__device__ void p2_issue(const ImgDesc &d, u32 q0, u32 n, int s, unsigned char *stages, P2Stage *st, u64 *full)
{
    // row of q0: a binary32 estimate (off by at most one) corrected exactly
    const u32 W = (u32)d.W;
    u32 y0 = (u32)__fmul_rz((float)q0, __frcp_rz((float)W));
    y0 = min(y0, (u32)d.H - 1u);
    while (y0 > 0 && y0 * W > q0) --y0;
    while ((y0 + 1u) * W <= q0) ++y0;
    const u32 x0 = q0 - y0 * W;
    const u32 na = min(n, W - x0);
    unsigned char *sb = stages + (size_t)s * kStageBytes;
    P2Stage &t = st[s];
    t.p0 = q0;
    t.n = (int)n;
    t.y0 = (int)y0;
    t.x0 = (int)x0;
    t.na = (int)na;
    t.fa = t.fb = -1;
    const u32 pbytes = (n * 8u + 15u) & ~15u;
    u32 abytes = 0, bbytes = 0;
    uintptr_t a0 = 0, b0 = 0;
    if (d.mode == MODE_HYBRID_EST && n - na <= (u32)d.W) {
        const uintptr_t ra = reinterpret_cast<uintptr_t>(d.fbuf + (size_t)y0 * d.f_pitch + (size_t)x0 * d.elem);
        a0 = ra & ~uintptr_t(15);
        abytes = (u32)(((ra + (size_t)na * d.elem + 15) & ~uintptr_t(15)) - a0);
        t.fa = kStagePlane + (int)(ra - a0);
        if (n > na) {
            b0 = reinterpret_cast<uintptr_t>(d.fbuf + (size_t)(y0 + 1) * d.f_pitch);
            bbytes = ((n - na) * (u32)d.elem + 15u) & ~15u;
            t.fb = kStagePlane + (int)abytes;
        }
    }
    mbar_expect_tx(&full[s], pbytes + abytes + bbytes);
    bulk_copy(sb, d.plane + 2 * (size_t)q0, pbytes, &full[s]);
    if (abytes) bulk_copy(sb + kStagePlane, reinterpret_cast<const void *>(a0), abytes, &full[s]);
    if (bbytes) bulk_copy(sb + kStagePlane + abytes, reinterpret_cast<const void *>(b0), bbytes, &full[s]);
}

// Row and column of pixel j of a unit (j >= na: the following rows).
__device__ __forceinline__ void unit_pixel(const ImgDesc &d, const P2Stage &t, u32 j, u32 &y, u32 &x)
{
    if (j < (u32)t.na) {
        y = (u32)t.y0;
        x = (u32)t.x0 + j;
    } else {
        const u32 r = j - (u32)t.na;
        if (r < (u32)d.W) {
            y = (u32)t.y0 + 1;
            x = r;
        } else {
            y = (u32)t.y0 + 1 + r / (u32)d.W;
            x = r % (u32)d.W;
        }
    }
}

// All threads: apply the staged unit (four pixels a thread).
__device__ void p2_apply(const ImgDesc &d, const unsigned char *sb, const P2Stage &t, float v2f)
{
    const u32 q0 = t.p0, n = (u32)t.n;
    const u32 j0 = threadIdx.x * 4u;
    if (j0 >= n) return;
    const int npx = (int)min(4u, n - j0);
    ApplyConst k;
    k.n = 0;
    k.v2f = v2f;
    k.inv_n = 0.f;
    k.inv_n2 = 0.f;
    k.maxv = (u32)d.maxv;
    const float4 *pp = reinterpret_cast<const float4 *>(sb) + 2 * threadIdx.x;
    const float4 m01 = pp[0], m23 = pp[1];
    const float mu[4] = {m01.x, m01.z, m23.x, m23.z};
    const float s2[4] = {m01.y, m01.w, m23.y, m23.w};
    const bool same_row = j0 + 3u < (u32)t.na || (j0 >= (u32)t.na && j0 + 3u - (u32)t.na < (u32)d.W);
    u32 fv[4], ov[4];
    float yv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        fv[i] = 0;
        if (i < npx) {
            const u32 j = j0 + i;
            if (t.fa >= 0) {
                const int off = j < (u32)t.na ? t.fa + (int)j * d.elem : t.fb + (int)(j - (u32)t.na) * d.elem;
                fv[i] = d.elem == 1 ? (u32)sb[off] : (u32)*reinterpret_cast<const u16 *>(sb + off);
            } else {
                const bool hyb = d.mode == MODE_HYBRID_EST;
                const uint8_t *fsrc = hyb ? d.fbuf : d.src;
                const long long fpitch = hyb ? d.f_pitch : d.src_pitch;
                u32 y, x;
                unit_pixel(d, t, j, y, x);
                const uint8_t *fp = fsrc + (long long)y * fpitch + (long long)x * d.elem;
                fv[i] = d.elem == 1 ? (u32)__ldcg(fp) : (u32)__ldcg(reinterpret_cast<const u16 *>(fp));
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) ov[i] = wiener_ms(mu[i], s2[i], fv[i], k, yv[i]);
    u32 y, x;
    unit_pixel(d, t, j0, y, x);
    uint8_t *op = d.dst + (long long)y * d.dst_pitch + (long long)x * d.elem;
    const uintptr_t oa = reinterpret_cast<uintptr_t>(op);
    if (npx == 4 && same_row && d.elem == 1 && (oa & 3) == 0) {
        *reinterpret_cast<u32 *>(op) = ov[0] | (ov[1] << 8) | (ov[2] << 16) | (ov[3] << 24);
    } else if (npx == 4 && same_row && d.elem == 2 && (oa & 7) == 0) {
        *reinterpret_cast<uint2 *>(op) = make_uint2(ov[0] | (ov[1] << 16), ov[2] | (ov[3] << 16));
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (i < npx) {
                u32 yy, xx;
                unit_pixel(d, t, j0 + i, yy, xx);
                uint8_t *o = d.dst + (long long)yy * d.dst_pitch + (long long)xx * d.elem;
                if (d.elem == 1) *o = (uint8_t)ov[i];
                else *reinterpret_cast<u16 *>(o) = (u16)ov[i];
            }
        }
    }
    if (d.y_out) {
        float *yp = d.y_out + q0 + j0;
        if (npx == 4 && (reinterpret_cast<uintptr_t>(yp) & 15) == 0) {
            *reinterpret_cast<float4 *>(yp) = make_float4(yv[0], yv[1], yv[2], yv[3]);
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (i < npx) yp[i] = yv[i];
        }
    }
}

// Wiener apply of one tile: vertical sliding sums of H1, H2 per column pair,
// two output pixels per lane and row, stored as one pixel pair.
template <bool NARROW>
__device__ void tile_apply(const ImgDesc &d, const Geo &g, const u16 *fs, u32 *H1, void *h2p, float v2f)
{
    const int w = d.w, wy = d.wh;      // window columns, rows
    // H1 and H2 are in place (run_item_t ran hsums, then a block barrier)
    ApplyConst k;
    k.n = (u32)(w * wy);
    k.v2f = v2f;
    k.inv_n = __frcp_rn((float)k.n);
    k.inv_n2 = __frcp_rn((float)(k.n * k.n));
    k.maxv = (u32)d.maxv;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x = 2 * lane;
    const int per = (g.th + kWarps - 1) / kWarps;
    const int j0 = warp * per, j1 = min(j0 + per, g.th);
    if (x >= g.tw || j0 >= j1) return;
    const bool two = x + 1 < g.tw;
    const u32 *H2n = reinterpret_cast<const u32 *>(h2p);
    const u64 *H2w = reinterpret_cast<const u64 *>(h2p);
    u32 sa = 0, sb = 0;
    u32 qa = 0, qb = 0;       // NARROW: S2 mod 2^32
    u64 wa = 0, wb = 0;       // WIDE
    for (int t = 0; t < wy; ++t) {
        const uint2 h = *reinterpret_cast<const uint2 *>(H1 + (j0 + t) * HS + x);
        sa += h.x;
        sb += h.y;
        if (NARROW) {
            const uint2 q = *reinterpret_cast<const uint2 *>(H2n + (j0 + t) * HS + x);
            qa += q.x;
            qb += q.y;
        } else {
            wa += H2w[(j0 + t) * HS + x];
            wb += H2w[(j0 + t) * HS + x + 1];
        }
    }
    for (int j = j0; j < j1; ++j) {
        float da, db;
        if (NARROW) {
            da = __uint2float_rn(k.n * qa - sa * sa);     // exact: the true value is < 2^32
            db = __uint2float_rn(k.n * qb - sb * sb);
        } else {
            da = __ull2float_rn((u64)k.n * wa - (u64)sa * sa);
            db = __ull2float_rn((u64)k.n * wb - (u64)sb * sb);
        }
        const u32 fp = *reinterpret_cast<const u32 *>(fs + (j + g.Ry) * FS + g.Lm + x);
        float ya, yb;
        const u32 oa = wiener_px(sa, da, fp & 0xffffu, k, ya);
        const u32 ob = wiener_px(sb, db, fp >> 16, k, yb);
        uint8_t *px = d.dst + (long long)(g.y0 + j) * d.dst_pitch + (long long)(g.x0 + x) * d.elem;
        if (d.elem == 1) {
            if (two && (reinterpret_cast<uintptr_t>(px) & 1) == 0) {
                *reinterpret_cast<u16 *>(px) = (u16)(oa | (ob << 8));
            } else {
                px[0] = (uint8_t)oa;
                if (two) px[1] = (uint8_t)ob;
            }
        } else {
            if (two && (reinterpret_cast<uintptr_t>(px) & 3) == 0) {
                *reinterpret_cast<u32 *>(px) = oa | (ob << 16);
            } else {
                reinterpret_cast<u16 *>(px)[0] = (u16)oa;
                if (two) reinterpret_cast<u16 *>(px)[1] = (u16)ob;
            }
        }
        if (d.y_out) {
            float *yp = d.y_out + (long long)(g.y0 + j) * d.W + g.x0 + x;
            yp[0] = ya;
            if (two) yp[1] = yb;
        }
        if (j + 1 < j1) {
            const uint2 hi_ = *reinterpret_cast<const uint2 *>(H1 + (j + wy) * HS + x);
            const uint2 ho_ = *reinterpret_cast<const uint2 *>(H1 + j * HS + x);
            sa += hi_.x - ho_.x;
            sb += hi_.y - ho_.y;
            if (NARROW) {
                const uint2 qi = *reinterpret_cast<const uint2 *>(H2n + (j + wy) * HS + x);
                const uint2 qo = *reinterpret_cast<const uint2 *>(H2n + j * HS + x);
                qa += qi.x - qo.x;
                qb += qi.y - qo.y;
            } else {
                wa += H2w[(j + wy) * HS + x];
                wa -= H2w[j * HS + x];
                wb += H2w[(j + wy) * HS + x + 1];
                wb -= H2w[j * HS + x + 1];
            }
        }
    }
}

// ---------------------------------------------------------------- one work item
struct Views {
    unsigned char *stage;     // plane-mode phase-2 stages (the whole dynamic area)
    u16 *fs, *gs, *wl0, *wl1;
    u32 *st_mm;
    u16 *st_c;
    u32 *h1;
    void *h2;
};

// One warp: the segment of ticket `item` (the last one with first <= item;
// the table is sorted by first) by a 32-way search, one ballot a round (two
// rounds for up to 1024 segments), into bs.seg[slot]; for batches also the
// image's descriptor, copied into bs.desc[slot].  Every thread of the CTA
// then reads both from shared memory instead of chasing the tables in
// global memory.
__device__ void resolve_item(const LaunchParams &lp, const Seg *segs, int item, BlockShared &bs, int slot)
{
    const int lane = threadIdx.x & 31;
    int stride = 1;
    while (stride * 32 < lp.nsegs) stride *= 32;
    int lo = 0;        // invariant: segs[lo].first <= item
    for (;;) {
        const int idx = lo + lane * stride;
        const bool le = idx < lp.nsegs && segs[idx].first <= item;
        const u32 b = __ballot_sync(FULL, le);      // a prefix of the lanes, lane 0 included
        lo += (31 - __clz(b)) * stride;
        if (stride == 1) break;
        stride >>= 5;
    }
    const Seg sg = segs[lo];
    if (lane == 0) bs.seg[slot] = sg;
    if (lp.descs) {
        const u32 *src = reinterpret_cast<const u32 *>(lp.descs + sg.img);
        u32 *dst = reinterpret_cast<u32 *>(&bs.desc[slot]);
        for (int i = lane; i < (int)(sizeof(ImgDesc) / 4); i += 32) dst[i] = src[i];
    }
}

__device__ __forceinline__ bool mode_median(int mode)
{
    return mode == MODE_AMF || mode == MODE_HYBRID_EST || mode == MODE_HYBRID_GIVEN;
}

// Tile geometry of an image with Wiener halo rw (0 for the median alone).
__device__ __forceinline__ void tile_shape(int rw, int ry, int FH, int &Lm, int &TW, int &TH)
{
    Lm = rw + (rw & 1);
    TW = (FW - Lm - rw) & ~1;
    TH = FH - 2 * ry;
}

// One work item.  Only the Wiener sums depend on `narrow` (32-bit sums exact):
// the median stages exist once per PACK, so a batch with both kinds of
// images does not run two copies of them (the instruction cache is a limit).
template <bool PACK>
__device__ void run_item_t(const ImgDesc &d, int phase, const Geo &g, const LaunchParams &lp, const Views &vw,
                           BlockShared &bs, bool narrow)
{
    const int mode = d.mode;
    const int FH = lp.region_h;
    const bool do_amf = phase == 1 && mode_median(mode);
    HD_STAMP_INIT();

    const bool est = mode == MODE_HYBRID_EST || mode == MODE_WIENER_EST;

    // ---- the region in shared memory, by one call site (one copy of the load
    // code): the noisy input with the median halo, or the f region (from the
    // median plane in a phase-2 item, else the input)
    {
        const bool fpl = !do_amf && phase == 2 && mode == MODE_HYBRID_EST;
        const uint8_t *base = fpl ? d.fbuf : d.src;
        const long long pitch = fpl ? d.f_pitch : d.src_pitch;
        const uint8_t *hi = fpl ? d.fbuf + (long long)d.H * d.f_pitch
                                : d.src + (long long)(d.H - 1) * d.src_pitch + (long long)d.W * d.elem;
        const int ra = do_amf ? g.Ra : 0;
        if (do_amf && threadIdx.x == 0) bs.cnt[0] = 0;
        load_region(do_amf ? vw.gs + g.pa : vw.fs, do_amf ? g.GS : FS, g.nrow + 2 * ra, g.ncol + 2 * ra, base, pitch,
                    d.elem, d.H, d.W, g.gfy - ra, g.gfx - ra, !do_amf && d.border_zero != 0, hi, fpl);
        __syncthreads();
    }
    if (do_amf) {
        HD_STAMP(0);
        if (PACK) amf3_packed(d, g, vw.gs, vw.fs, vw.wl0, &bs.cnt[0], FH);
        else amf3_scalar(d, g, vw.gs, vw.fs, vw.wl0, &bs.cnt[0], FH);
        __syncthreads();
        HD_STAMP(1);
        if (d.smax > 3)
            amf_grow<PACK>(d, g, vw.gs, vw.fs, vw.wl0, vw.wl1, bs.cnt, FH * FW, vw.st_mm, vw.st_c,
                           lp.small_growth, lp.select_lanes);
        if ((g.Rw > 0 || g.Ry > 0) && d.border_zero) {
            // zero-border Wiener: samples outside the image read 0 (after every
            // growth write: the short-worklist path ends without a barrier)
            __syncthreads();
            for (int i = threadIdx.x; i < g.nrow * g.ncol; i += kThreads) {
                const int r = i / g.ncol, c = i - r * g.ncol;
                const int gy = g.gfy + r, gx = g.gfx + c;
                if ((unsigned)gy >= (unsigned)d.H || (unsigned)gx >= (unsigned)d.W) vw.fs[r * FS + c] = 0;
            }
        }
        __syncthreads();
    } else {
        HD_STAMP(5);
    }
    if (do_amf) HD_STAMP(2);

    // the median output: the result (median only) or the median plane (one call site)
    const bool amf_only = mode == MODE_AMF;
    if (amf_only || (phase == 1 && mode == MODE_HYBRID_EST)) {
        store_region(vw.fs + g.Ry * FS + g.Lm, FS, g.th, g.tw, amf_only ? d.dst : d.fbuf,
                     amf_only ? d.dst_pitch : d.f_pitch, d.elem, g.y0, g.x0);
        if (amf_only) return;
        HD_STAMP(3);
    }
    // the horizontal window sums of the f region, by one call site per sum
    // width (the statistics pass needs H2 only for the plane)
    {
        const bool with_h2 = !(phase == 1 && est) || d.plane != nullptr;
        if (PACK && narrow) hsums<true>(g, vw.fs, vw.h1, vw.h2, d.w, with_h2);
        else hsums<false>(g, vw.fs, vw.h1, vw.h2, d.w, with_h2);
    }
    if (phase == 1 && est) {
        if (PACK && narrow) {
            if (d.plane) tile_stats<true, true>(d, g, vw.fs, vw.h1, vw.h2, bs);
            else tile_stats<true, false>(d, g, vw.fs, vw.h1, vw.h2, bs);
        } else {
            if (d.plane) tile_stats<false, true>(d, g, vw.fs, vw.h1, vw.h2, bs);
            else tile_stats<false, false>(d, g, vw.fs, vw.h1, vw.h2, bs);
        }
        HD_STAMP(4);
        return;
    }
    // one thread converts the noise variance (binary64 is slow here); the
    // value is cached per CTA for the image's following tiles
    if (threadIdx.x == 0) {
        if (!est || bs.nu2_of != d.ctl) {
            const u64 n = (u64)d.w * (u64)d.wh;
            const double nu2 = est ? noise_variance(d.ctl, n, d.Hg, d.W, d.inv_den) : d.noise_var;
            bs.nu2 = nu2;
            bs.nu2f = __double2float_rn(nu2);
            bs.nu2_of = est ? d.ctl : nullptr;
        }
        if (g.x0 == 0 && g.y0 == 0 && d.noise_var_out) *d.noise_var_out = bs.nu2;
    }
    __syncthreads();
    if (PACK && narrow) tile_apply<true>(d, g, vw.fs, vw.h1, vw.h2, bs.nu2f);
    else tile_apply<false>(d, g, vw.fs, vw.h1, vw.h2, bs.nu2f);
    HD_STAMP(6);
}

// Plane-mode phase 2 read straight from L2: the CTA's share of image d is
// pixels [pb, pe) of the row-major order (the gridDim.x shares equal up to a
// pixel pair, each starting an even distance after the first owned pixel, so
// that a group's (mu, s2) pairs start on a 16-byte boundary).  Thread t
// applies the 4-pixel groups t, t + kThreads, ... of the share; the loads of
// a thread's next group are issued before the arithmetic of its current one,
// and no block barrier is taken after the noise variance is known.
struct P2Group {
    float4 a, b;      // (mu, s2) of pixels 0, 1 and of pixels 2, 3
    u32 f[4];         // f of the four pixels
};

__device__ __forceinline__ void p2_locate(u64 q, u32 W, u32 &y, u32 &x)
{
    y = (u32)(q / W);
    x = (u32)(q - (u64)y * W);
}

__device__ __forceinline__ void p2_load(const ImgDesc &d, const uint8_t *fsrc, long long fpitch, u64 q, u32 y,
                                        u32 x, u32 n, P2Group &g)
{
    const u32 W = (u32)d.W;
    const float2 *pp = reinterpret_cast<const float2 *>(d.plane) + q;
    const uint8_t *fp = fsrc + (long long)y * fpitch + (long long)x * d.elem;
    const uintptr_t fa = reinterpret_cast<uintptr_t>(fp);
    if (n == 4 && x + 4u <= W && (d.elem == 1 ? (fa & 3) == 0 : (fa & 7) == 0)) {
        g.a = __ldcg(reinterpret_cast<const float4 *>(pp));
        g.b = __ldcg(reinterpret_cast<const float4 *>(pp) + 1);
        if (d.elem == 1) {
            const u32 v = __ldcg(reinterpret_cast<const unsigned int *>(fp));
            g.f[0] = v & 0xffu;
            g.f[1] = (v >> 8) & 0xffu;
            g.f[2] = (v >> 16) & 0xffu;
            g.f[3] = v >> 24;
        } else {
            const uint2 v = __ldcg(reinterpret_cast<const uint2 *>(fp));
            g.f[0] = v.x & 0xffffu;
            g.f[1] = v.x >> 16;
            g.f[2] = v.y & 0xffffu;
            g.f[3] = v.y >> 16;
        }
        return;
    }
    float m[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    u32 yy = y, xx = x;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        g.f[i] = 0;
        if ((u32)i < n) {
            const float2 v = __ldcg(pp + i);
            m[2 * i] = v.x;
            m[2 * i + 1] = v.y;
            const uint8_t *p = fsrc + (long long)yy * fpitch + (long long)xx * d.elem;
            g.f[i] = d.elem == 1 ? (u32)__ldcg(p) : (u32)__ldcg(reinterpret_cast<const u16 *>(p));
            if (++xx == W) {
                xx = 0;
                ++yy;
            }
        }
    }
    g.a = make_float4(m[0], m[1], m[2], m[3]);
    g.b = make_float4(m[4], m[5], m[6], m[7]);
}

__device__ __forceinline__ void p2_store(const ImgDesc &d, u64 q, u32 y, u32 x, u32 n, const P2Group &g,
                                         const ApplyConst &k)
{
    const u32 W = (u32)d.W;
    u32 o[4];
    float yv[4];
    o[0] = wiener_ms(g.a.x, g.a.y, g.f[0], k, yv[0]);
    o[1] = wiener_ms(g.a.z, g.a.w, g.f[1], k, yv[1]);
    o[2] = wiener_ms(g.b.x, g.b.y, g.f[2], k, yv[2]);
    o[3] = wiener_ms(g.b.z, g.b.w, g.f[3], k, yv[3]);
    uint8_t *op = d.dst + (long long)y * d.dst_pitch + (long long)x * d.elem;
    const uintptr_t oa = reinterpret_cast<uintptr_t>(op);
    if (n == 4 && x + 4u <= W && d.elem == 1 && (oa & 3) == 0) {
        *reinterpret_cast<u32 *>(op) = o[0] | (o[1] << 8) | (o[2] << 16) | (o[3] << 24);
    } else if (n == 4 && x + 4u <= W && d.elem == 2 && (oa & 7) == 0) {
        *reinterpret_cast<uint2 *>(op) = make_uint2(o[0] | (o[1] << 16), o[2] | (o[3] << 16));
    } else {
        u32 yy = y, xx = x;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if ((u32)i < n) {
                uint8_t *p = d.dst + (long long)yy * d.dst_pitch + (long long)xx * d.elem;
                if (d.elem == 1) *p = (uint8_t)o[i];
                else *reinterpret_cast<u16 *>(p) = (u16)o[i];
                if (++xx == W) {
                    xx = 0;
                    ++yy;
                }
            }
        }
    }
    if (d.y_out) {
        float *yp = d.y_out + q;
        if (n == 4 && (reinterpret_cast<uintptr_t>(yp) & 15) == 0) {
            *reinterpret_cast<float4 *>(yp) = make_float4(yv[0], yv[1], yv[2], yv[3]);
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if ((u32)i < n) yp[i] = yv[i];
        }
    }
}

__device__ void p2_direct(const ImgDesc &d, const LaunchParams &lp, BlockShared &bs)
{
    HD_STAMP_INIT();
    if (!wait_phase1(d, (u32)(d.tiles_x * d.tiles_y), lp.spin_limit, &bs.flag)) return;
    HD_STAMP(12);
    const u64 P0 = (u64)d.own0 * (u64)d.W, NP = (u64)(d.own1 - d.own0) * (u64)d.W;
    const u64 per = ((NP + 1) / 2 + gridDim.x - 1) / gridDim.x;     // pixel pairs per CTA
    const u64 pb = P0 + min(NP, 2 * per * blockIdx.x), pe = P0 + min(NP, 2 * per * (blockIdx.x + 1));
    const bool hyb = d.mode == MODE_HYBRID_EST;
    const uint8_t *fsrc = hyb ? d.fbuf : d.src;
    const long long fpitch = hyb ? d.f_pitch : d.src_pitch;
    const u32 W = (u32)d.W;
    constexpr u32 kStep = 4u * kThreads;
    // the first group's loads go out while thread 0 converts the noise variance
    u64 q = pb + 4u * threadIdx.x;
    u32 y = 0, x = 0;
    P2Group cur;
    if (q < pe) {
        p2_locate(q, W, y, x);
        p2_load(d, fsrc, fpitch, q, y, x, (u32)min((u64)4, pe - q), cur);
    }
    if (threadIdx.x == 0) {
        const double nu2 = noise_variance(d.ctl, (u64)d.w * (u64)d.wh, d.Hg, d.W, d.inv_den);
        bs.nu2 = nu2;
        bs.nu2f = __double2float_rn(nu2);
        if (blockIdx.x == 0 && d.noise_var_out) *d.noise_var_out = nu2;
    }
    __syncthreads();
    HD_STAMP(21);
    ApplyConst k;
    k.n = 0;
    k.v2f = bs.nu2f;
    k.inv_n = 0.f;
    k.inv_n2 = 0.f;
    k.maxv = (u32)d.maxv;
    while (q < pe) {
        const u32 n = (u32)min((u64)4, pe - q);
        const u64 qn = q + kStep;
        u32 yn = y, xn = x + kStep;
        while (xn >= W) {
            xn -= W;
            ++yn;
        }
        P2Group nxt;
        if (qn < pe) p2_load(d, fsrc, fpitch, qn, yn, xn, (u32)min((u64)4, pe - qn), nxt);
        p2_store(d, q, y, x, n, cur, k);
        cur = nxt;
        q = qn;
        y = yn;
        x = xn;
    }
    HD_STAMP(20);
}

// Plane-mode phase 2 of the CTA's share of image d: pixels [pb, pe), the
// gridDim.x shares being equal up to a pixel pair.
__device__ void p2_share(const ImgDesc &d, const LaunchParams &lp, const Views &vw, BlockShared &bs)
{
    HD_STAMP_INIT();
    if (!wait_phase1(d, (u32)(d.tiles_x * d.tiles_y), lp.spin_limit, &bs.flag)) return;
    HD_STAMP(12);
    HD_CTA_T(2);
    // the plane and f rows were written by other CTAs (generic stores, made
    // visible by the wait); the bulk copies read them through the async proxy
    if (threadIdx.x < kStages) asm volatile("fence.proxy.async.global;" ::: "memory");
    // the owned pixels [P0, P1) (the whole image unless it is a part), in
    // shares starting P0 + an even offset: with the plane base placed so that
    // pixel P0's pair is 16-byte aligned, every unit's pairs are too
    const u64 P0 = (u64)d.own0 * (u64)d.W, NP = (u64)(d.own1 - d.own0) * (u64)d.W;
    const u64 per = ((NP + 1) / 2 + gridDim.x - 1) / gridDim.x;     // pixel pairs per CTA
    const u32 pb = (u32)(P0 + min(NP, 2 * per * blockIdx.x)), pe = (u32)(P0 + min(NP, 2 * per * (blockIdx.x + 1)));
    // K units of one even size (the last one takes the remainder): every unit
    // starts inside the share
    const u32 S = pe - pb, K0 = (S + kUnitPx - 1) / kUnitPx;
    const u32 usz = K0 > 0 ? min((u32)kUnitPx, ((S + K0 - 1) / K0 + 1) & ~1u) : 1u;
    const int K = (int)((S + usz - 1) / usz);
    // priming: lanes 0..kStages-1 of warp 0 stage one unit each; a thread of
    // warp 1 converts the noise variance meanwhile
    if (threadIdx.x < kStages) {
        const int st = threadIdx.x;
        // generic writes to the stage area (phase-1 work) are ordered before
        // the async copies into it; later a stage is refilled only after the
        // block barrier that ends its reads
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (st < K) {
            const u32 q = pb + (u32)st * usz;
            p2_issue(d, q, min(usz, pe - q), st, vw.stage, bs.st, bs.full);
        } else {
            bs.st[st].n = 0;
        }
    }
    if (threadIdx.x == 32) {
        const double nu2 = noise_variance(d.ctl, (u64)d.w * (u64)d.wh, d.Hg, d.W, d.inv_den);
        bs.nu2 = nu2;
        bs.nu2f = __double2float_rn(nu2);
        if (blockIdx.x == 0 && d.noise_var_out) *d.noise_var_out = nu2;
    }
    __syncthreads();
    HD_STAMP(21);
    for (int k = 0; k < K; ++k) {
        const int st = k % kStages;
        const bool late = !mbar_wait(&bs.full[st], (bs.fullpar >> st) & 1u, lp.spin_limit);
        HD_STAMP(19);
        p2_apply(d, vw.stage + (size_t)st * kStageBytes, bs.st[st], bs.nu2f);
        HD_STAMP(20);
        if (__syncthreads_or(late)) {
            // a copy did not land in time: report, wait (bounded) for the
            // copies still in flight, and give up the share
            if (threadIdx.x == 0) {
                atomicOr(&g_device_error, DEVERR_TIMEOUT);
                for (int j = 0; j < kStages; ++j) {
                    const int sj = (k + j) % kStages;
                    if (bs.st[sj].n > 0) {
                        mbar_wait(&bs.full[sj], (bs.fullpar >> sj) & 1u, lp.spin_limit);
                        bs.fullpar ^= 1u << sj;
                    }
                    bs.st[sj].n = 0;
                }
            }
            __syncthreads();
            return;
        }
        if (threadIdx.x == 0) {
            bs.fullpar ^= 1u << st;
            const int kn = k + kStages;
            if (kn < K) {
                const u32 q = pb + (u32)kn * usz;
                p2_issue(d, q, min(usz, pe - q), st, vw.stage, bs.st, bs.full);
            } else {
                bs.st[st].n = 0;
            }
        }
        HD_STAMP(22);
    }
    HD_STAMP(13);
}

__device__ __forceinline__ bool image_narrow(const ImgDesc &d)
{
    const long long n = (long long)d.w * d.wh;
    return d.maxv < 0x8000 && (long long)(max(d.w, d.wh) + 1) * d.maxv <= 65535 && n * d.maxv < 131072;
}

__device__ void run_item(const ImgDesc &d, int phase, int tile, const LaunchParams &lp, const Views &vw,
                         BlockShared &bs)
{
    Geo g;
    g.Rw = d.mode == MODE_AMF ? 0 : (d.w >> 1);
    g.Ry = d.mode == MODE_AMF ? 0 : (d.wh >> 1);
    int TW, TH;
    tile_shape(g.Rw, g.Ry, lp.region_h, g.Lm, TW, TH);
    g.hx = g.Lm - g.Rw;
    g.Ra = (phase == 1 && mode_median(d.mode)) ? (d.smax >> 1) : 0;
    g.pa = g.Ra & 1;
    g.GS = g_stride(g.Ra);
    const int tyi = tile / d.tiles_x, txi = tile - tyi * d.tiles_x;
    g.x0 = txi * TW;
    g.y0 = d.own0 + tyi * TH;
    g.tw = min(TW, d.W - g.x0);
    g.th = min(TH, d.own1 - g.y0);
    g.ncol = g.Lm + g.tw + g.Rw;
    g.nrow = g.th + 2 * g.Ry;
    g.gfx = g.x0 - g.Lm;
    g.gfy = g.y0 - g.Ry;

    if (phase == 2 && bs.nu2_of != d.ctl) {
        HD_STAMP_INIT();
        const bool ok = wait_phase1(d, (u32)(d.tiles_x * d.tiles_y), lp.spin_limit, &bs.flag);
        HD_STAMP(7);
        if (!ok) return;
    }
    const bool pack = d.maxv < 0x8000;
    const bool narrow = image_narrow(d);
#ifdef HD_STAGE_PROFILE
    const long long tc0 = clock64();
#endif
    if (pack) run_item_t<true>(d, phase, g, lp, vw, bs, narrow);
    else run_item_t<false>(d, phase, g, lp, vw, bs, false);
#ifdef HD_STAGE_PROFILE
    if (threadIdx.x == 0 && phase == 1 && tile < (1 << 16)) g_tile_cyc[tile] = (unsigned int)(clock64() - tc0);
#endif
}

__global__ void __launch_bounds__(kThreads, 4) hd_persistent_kernel(const __grid_constant__ LaunchParams lp)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ BlockShared bs;
    const SmemLayout L = layout(lp.region_h, lp.ra_max, lp.wide);
    Views vw;
    vw.stage = smem_raw;
    vw.fs = reinterpret_cast<u16 *>(smem_raw + L.fs);
    vw.gs = reinterpret_cast<u16 *>(smem_raw + L.gs);
    vw.wl0 = reinterpret_cast<u16 *>(smem_raw + L.wl);
    vw.wl1 = vw.wl0 + lp.region_h * FW;
    vw.st_mm = reinterpret_cast<u32 *>(smem_raw + L.st);
    vw.st_c = reinterpret_cast<u16 *>(smem_raw + L.st + (size_t)lp.region_h * FW * sizeof(u32));
    vw.h1 = reinterpret_cast<u32 *>(smem_raw + L.h1);
    vw.h2 = smem_raw + L.h2;

    const Seg *segs = lp.segs ? lp.segs : lp.oneseg;
    HD_STAMP_INIT();
    HD_CTA_T(0);
#ifdef HD_STAGE_PROFILE
    int nitems = 0;
#endif
    int buf = 0;
    int item;
    if (threadIdx.x == 0) {
        bs.nu2_of = nullptr;
        bs.fullpar = 0;
        for (int i = 0; i < kStages; ++i) mbar_init(&bs.full[i], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // the first item: its ticket and, with tables (batches), its segment and
    // descriptor, resolved by the last warp (thread 0 ends a median item with
    // the sums' atomics and the release of its done count, so the two waits
    // overlap); a single image has at most two segments in the launch
    // parameters
    const bool tables = lp.segs != nullptr;
    const bool rwarp = (threadIdx.x >> 5) == kWarps - 1, rlead = threadIdx.x == kThreads - 32;
    if (rwarp) {
        int first = 0;
        if (rlead) first = lp.ticket ? (int)atomicAdd(lp.ticket, 1u) : (int)blockIdx.x;
        first = __shfl_sync(FULL, first, 0);
        if (rlead) bs.item[0] = first;
        if (tables && first < lp.total_items) resolve_item(lp, segs, first, bs, 0);
    }
    __syncthreads();
    item = bs.item[0];
    while (item < lp.total_items) {
        const Seg sg = tables ? bs.seg[buf]
                              : (lp.nsegs > 1 && item >= lp.oneseg[1].first ? lp.oneseg[1] : lp.oneseg[0]);
        const ImgDesc &d = lp.descs ? bs.desc[buf] : lp.one;
        // Take the next ticket now and read it after the item: its latency
        // hides behind the work.  Tickets only grow, and an item waits only on
        // earlier tickets, so the CTA holding the earliest unfinished ticket
        // is always working on it: holding a later one cannot deadlock.
        int next = 0;
        if (rlead) next = lp.ticket ? (int)atomicAdd(lp.ticket, 1u) : item + (int)gridDim.x;
        run_item(d, sg.phase, item - sg.first, lp, vw, bs);
#ifdef HD_STAGE_PROFILE
        ++nitems;
#endif
        // the last warp resolves the next item into the other slot (the
        // current slot stays valid until the barrier)
        if (rwarp) {
            next = __shfl_sync(FULL, next, 0);
            if (rlead) bs.item[buf ^ 1] = next;
            if (tables && next < lp.total_items) resolve_item(lp, segs, next, bs, buf ^ 1);
        }
        __syncthreads();
        buf ^= 1;
        item = bs.item[buf];
    }
    HD_STAMP(14);
    HD_CTA_T(1);
    HD_CTA_ITEMS(nitems);
    // plane mode: every CTA applies its share of the image's phase 2
    if (lp.p2_plane) {
        if (lp.p2_direct) p2_direct(lp.one, lp, bs);
        else p2_share(lp.one, lp, vw, bs);
    }
    HD_CTA_T(3);
    // The last CTA out leaves the queue counters and control blocks zeroed
    // for the next launch on this workspace.
    if (lp.ticket && threadIdx.x == 0) {
        __threadfence();
        const u32 done = atomicAdd(lp.ticket + 1, 1u);
        if (done == gridDim.x - 1) {
            __threadfence();
            for (int i = 0; i < lp.nctl; ++i) {
                ImgCtl &c = lp.ctl_reset[i];
                c.A_lo32 = 0;
                c.A_hi32 = 0;
                c.B_lo32 = 0;
                c.B_hi32 = 0;
                c.p1_done = 0;
            }
            lp.ticket[0] = 0;
            lp.ticket[1] = 0;
            __threadfence();
        }
    }
}

// Copies a chunk of a host-built table, carried in the kernel parameters, to
// device memory: table uploads need no host-side copy and no stream sync.
struct TableChunk {
    unsigned char *dst;
    unsigned int n;
    unsigned char bytes[kTableChunkBytes];
};

__global__ void hd_table_writer(const __grid_constant__ TableChunk c)
{
    for (unsigned int i = threadIdx.x; i < c.n; i += blockDim.x) c.dst[i] = c.bytes[i];
}

}  // namespace

int launch_table_upload(void *dst, const void *src, size_t bytes, void *stream)
{
    static_assert(sizeof(TableChunk) <= 32000, "kernel parameter limit");
    const unsigned char *s = static_cast<const unsigned char *>(src);
    for (size_t off = 0; off < bytes; off += kTableChunkBytes) {
        const size_t n = bytes - off < (size_t)kTableChunkBytes ? bytes - off : (size_t)kTableChunkBytes;
        TableChunk c;
        c.dst = static_cast<unsigned char *>(dst) + off;
        c.n = (unsigned int)n;
        memcpy(c.bytes, s + off, n);
        hd_table_writer<<<1, 256, 0, (cudaStream_t)stream>>>(c);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return (int)e;
    }
    return 0;
}

size_t smem_bytes(int region_h, int ra_max, int wide)
{
    return layout(region_h, ra_max, wide).total;
}

// The kernel's dynamic shared-memory limit only ever grows to the largest
// size requested so far: launches and occupancy queries of smaller sizes stay
// valid under it.
static std::mutex g_attr_mu;
static size_t g_attr_bytes = 48 * 1024;

static cudaError_t ensure_smem_limit(size_t smem)
{
    std::lock_guard<std::mutex> lk(g_attr_mu);
    if (smem <= g_attr_bytes) return cudaSuccess;
    const cudaError_t e =
        cudaFuncSetAttribute(hd_persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) g_attr_bytes = smem;
    return e;
}

int launch_persistent(const LaunchParams &lp, int grid, size_t smem, void *stream)
{
    const cudaError_t e = ensure_smem_limit(smem);
    if (e != cudaSuccess) return (int)e;
    hd_persistent_kernel<<<grid, kThreads, smem, (cudaStream_t)stream>>>(lp);
    return (int)cudaGetLastError();
}

int max_ctas_per_sm(size_t smem)
{
    // occupancy per shared-memory size, cached (the query is not free)
    static std::mutex mu;
    static size_t keys[16];
    static int vals[16];
    static int used = 0;
    std::lock_guard<std::mutex> lk(mu);
    for (int i = 0; i < used; ++i)
        if (keys[i] == smem) return vals[i];
    if (ensure_smem_limit(smem) != cudaSuccess) return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, hd_persistent_kernel, kThreads, smem) != cudaSuccess)
        return 0;
    if (used < 16) {
        keys[used] = smem;
        vals[used] = n;
        ++used;
    }
    return n;
}

int sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return n;
}

#ifdef HD_STAGE_PROFILE
extern "C" int hd_debug_tile_cycles(unsigned int *out, int n)
{
    return (int)cudaMemcpyFromSymbol(out, g_tile_cyc, (size_t)n * sizeof(unsigned int));
}

extern "C" int hd_debug_cta_times(unsigned long long *out, int n)
{
    return (int)cudaMemcpyFromSymbol(out, g_cta_t, (size_t)n * 5 * sizeof(unsigned long long));
}

extern "C" int hd_debug_stage_cycles(unsigned long long *out16, int clear)
{
    cudaError_t e = cudaMemcpyFromSymbol(out16, g_stage_cycles, 32 * sizeof(unsigned long long));
    if (e == cudaSuccess && clear) {
        unsigned long long z[32] = {0};
        e = cudaMemcpyToSymbol(g_stage_cycles, z, sizeof(z));
    }
    return (int)e;
}
#endif

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
