// hd_fft.cu -- the Wiener filter in the Fourier domain (Section IV places the
// hybrid's Wiener stage there): deconvolution of the image by a point-spread
// function P with a noise-to-signal ratio nsr,
//   F(u, v) = conj(P(u, v)) / (|P(u, v)|^2 + nsr) * G(u, v),  y = Re IDFT(F),
// with the 2-D DFT's periodic extension as the border rule and
// out = min(maxv, floor(y + 1/2)) (negatives to 0).
//
// The 2-D DFT is a row pass and a column pass of 1-D DFTs.  A CTA transforms
// 8192 / M rows at once, each held whole in shared memory (binary32 complex),
// with the twiddles staged in shared memory per stage:
//   - a power-of-two length M: radix-2 in place, decimation in time from
//     bit-reversed input to natural output (forward and inverse alike;
//     the inverse conjugates the twiddles);
//   - any other length N <= 4096: Bluestein's chirp-z method (L. Bluestein,
//     IEEE Trans. Audio Electroacoust. 18(4), 1970): with w_k = exp(-pi i
//     k^2 / N), X_k = w_k sum_n (x_n w_n) conj(w_{k-n}), a circular
//     convolution of length M = the power of two >= 2N - 1, done as a
//     forward radix-2 transform, a product with the precomputed transform
//     of the chirp, and an inverse transform by decimation in frequency
//     (natural input, bit-reversed output).
// Columns become rows by a tiled transpose.  The column pass of the image
// does the forward DFT, the product with the filter and the inverse DFT of
// the column in one CTA.  Twiddles and chirps are computed once per call in
// binary64 (sincospi) and rounded to binary32.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "hybrid_denoise.h"

namespace {

typedef unsigned int u32;
typedef unsigned short u16;

constexpr int kFftThreads = 1024;
constexpr int kMaxM = 8192;                   // longest transform held in shared memory
constexpr int kStageElems = kMaxM / kFftThreads;
constexpr size_t kAlign = 256;

inline size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Tables of one row length N.
struct LenTables {
    int N, M, logM;         // M = N (a power of two) or the Bluestein length
    const float2 *tw;       // M/2 entries: exp(-2 pi i k / M)
    const float2 *chirp;    // N entries: exp(-pi i k^2 / N) (Bluestein only)
    const float2 *bhat;     // M entries: forward DFT_M of b, b_m = conj(chirp_|m|) (Bluestein only)
};

enum Load { LOAD_IMAGE = 0, LOAD_PSF = 1, LOAD_COMPLEX = 2 };
enum Op { OP_FWD = 0, OP_INV = 1, OP_FILTER = 2 };
enum Store { STORE_COMPLEX = 0, STORE_IMAGE = 1 };

struct RowParams {
    LenTables t;
    int rows;
    int load, op, store;
    // LOAD_IMAGE: the image rows (real values)
    const uint8_t *img;
    long long img_pitch;
    int elem;
    // LOAD_PSF: row r of the PSF placed on a grid of grid_rows rows and N
    // columns with its centre tap at the origin, taps wrapped around
    const float *psf;
    int kh, kw, grid_rows;
    // LOAD_COMPLEX
    const float2 *in;
    long long in_stride;
    // OP_FILTER: rows of the PSF's transfer function, same layout as `in`
    const float2 *pspec;
    long long pspec_stride;
    float nsr;
    // STORE_COMPLEX
    float2 *out;
    long long out_stride;
    // STORE_IMAGE: y = Re(x) * scale; out = min(maxv, floor(y + 1/2))
    uint8_t *dst;
    long long dst_pitch;
    float scale;
    u32 maxv;
    float *y_out;           // optional, row stride N floats
};

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ int bitrev(int k, int logM) { return (int)(__brev((u32)k) >> (32 - logM)); }

// Radix-2 decimation in time: bit-reversed input, natural output.  The
// butterfly of span h at position p uses exp(-+2 pi i p / (2h)), which sits
// at ts[h - 1 + p] of the per-stage table in shared memory (consecutive
// positions at consecutive entries: no bank conflicts).  lt and T: this
// thread's index within its row group and the group's size.
__device__ void fft_dit(float2 *x, int M, int logM, const float2 *ts, bool inverse, int lt, int T)
{
    for (int s = 1; s <= logM; ++s) {
        const int half = 1 << (s - 1);
        for (int b = lt; b < (M >> 1); b += T) {
            const int pos = b & (half - 1);
            const int i = ((b >> (s - 1)) << s) + pos, j = i + half;
            float2 w = ts[half - 1 + pos];
            if (inverse) w.y = -w.y;
            const float2 u = x[i], v = cmul(w, x[j]);
            x[i] = make_float2(u.x + v.x, u.y + v.y);
            x[j] = make_float2(u.x - v.x, u.y - v.y);
        }
        __syncthreads();
    }
}

// Radix-2 decimation in frequency: natural input, bit-reversed output.
__device__ void fft_dif(float2 *x, int M, int logM, const float2 *ts, bool inverse, int lt, int T)
{
    for (int s = logM; s >= 1; --s) {
        const int half = 1 << (s - 1);
        for (int b = lt; b < (M >> 1); b += T) {
            const int pos = b & (half - 1);
            const int i = ((b >> (s - 1)) << s) + pos, j = i + half;
            float2 w = ts[half - 1 + pos];
            if (inverse) w.y = -w.y;
            const float2 u = x[i], v = x[j];
            x[i] = make_float2(u.x + v.x, u.y + v.y);
            x[j] = cmul(w, make_float2(u.x - v.x, u.y - v.y));
        }
        __syncthreads();
    }
}

// x[k] -> x[bitrev(k)] for k < M, through registers (every thread holds at
// most kStageElems entries).
__device__ void bitrev_inplace(float2 *x, int M, int logM, int lt, int T)
{
    float2 v[kStageElems];
#pragma unroll
    for (int i = 0; i < kStageElems; ++i) {
        const int k = lt + i * T;
        if (k < M) v[i] = x[k];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kStageElems; ++i) {
        const int k = lt + i * T;
        if (k < M) x[bitrev(k, logM)] = v[i];
    }
    __syncthreads();
}

// Unscaled DFT of x[0, N) in shared memory, in place, natural order in and
// out: sum_n x_n exp(-+2 pi i n k / N) (sign + for the inverse); ts is the
// per-stage twiddle table of t.M in shared memory (see fft_dit).
__device__ void dft_row(float2 *x, const LenTables &t, const float2 *ts, bool inverse, int lt, int T)
{
    const int N = t.N, M = t.M, logM = t.logM;
    if (M == 1) return;
    if (M == N) {
        bitrev_inplace(x, M, logM, lt, T);
        fft_dit(x, M, logM, ts, inverse, lt, T);
        return;
    }
    // Bluestein; the inverse through conjugation: IDFT(x) = conj(DFT(conj(x)))
    float2 v[kStageElems];
#pragma unroll
    for (int i = 0; i < kStageElems; ++i) {
        const int k = lt + i * T;
        float2 a = make_float2(0.f, 0.f);
        if (k < N) {
            a = x[k];
            if (inverse) a.y = -a.y;
            a = cmul(a, __ldg(&t.chirp[k]));
        }
        v[i] = a;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kStageElems; ++i) {
        const int k = lt + i * T;
        if (k < M) x[bitrev(k, logM)] = v[i];
    }
    __syncthreads();
    fft_dit(x, M, logM, ts, false, lt, T);
    for (int k = lt; k < M; k += T) x[k] = cmul(x[k], __ldg(&t.bhat[k]));
    __syncthreads();
    fft_dif(x, M, logM, ts, true, lt, T);
    // X_k = w_k c_k / M, c in bit-reversed order
#pragma unroll
    for (int i = 0; i < kStageElems; ++i) {
        const int k = lt + i * T;
        if (k < N) v[i] = x[bitrev(k, logM)];
    }
    __syncthreads();
    const float inv_m = 1.0f / (float)M;
#pragma unroll
    for (int i = 0; i < kStageElems; ++i) {
        const int k = lt + i * T;
        if (k < N) {
            float2 r = cmul(v[i], __ldg(&t.chirp[k]));
            r.x *= inv_m;
            r.y *= inv_m;
            if (inverse) r.y = -r.y;
            x[k] = r;
        }
    }
    __syncthreads();
}

// Rows per CTA for a transform length M: the CTA's 1024 threads split into
// groups of 1024 / R, each transforming one row in its own M entries of
// shared memory (R M <= kMaxM, so every thread stages at most kStageElems).
__host__ __device__ inline int rows_per_cta(int M) { return M >= kMaxM ? 1 : (kMaxM / M < 64 ? kMaxM / M : 64); }

// R rows per CTA (grid-stride over row groups): load, transform, store.
// Every group runs the same transform (same length and operation).  A group
// can be narrower than a warp, so one warp may hold a row and a group past
// the last row: every block-wide barrier therefore sits where all threads of
// the CTA reach it, behind conditions that are the same for the whole CTA.
// A group past the last row transforms zeros and stores nothing.
__global__ void __launch_bounds__(kFftThreads) fft_rows_kernel(const __grid_constant__ RowParams p)
{
    extern __shared__ float2 xs_all[];
    const int N = p.t.N, M = p.t.M;
    const int R = rows_per_cta(M), T = kFftThreads / R;
    const int grp = threadIdx.x / T, lt = threadIdx.x - grp * T;
    float2 *xs = xs_all + (size_t)grp * M;
    // the per-stage twiddle table: stage s (span h = 2^(s-1)) holds
    // exp(-2 pi i p / (2h)) = tw[p M / (2h)] for p < h at entries h - 1 + p
    float2 *ts = xs_all + (size_t)R * M;
    for (int e = threadIdx.x; e < M - 1; e += blockDim.x) {
        const int h = 1 << (31 - __clz(e + 1));
        ts[e] = __ldg(&p.t.tw[(e + 1 - h) * (M / (2 * h))]);
    }
    __syncthreads();
    for (int r0 = blockIdx.x * R; r0 < p.rows; r0 += gridDim.x * R) {
        const int r = r0 + grp;
        const bool live = r < p.rows;
        if (p.load == LOAD_PSF || !live)
            for (int k = lt; k < N; k += T) xs[k] = make_float2(0.f, 0.f);
        if (p.load == LOAD_PSF) __syncthreads();
        if (live) {
            if (p.load == LOAD_IMAGE) {
                const uint8_t *row = p.img + (long long)r * p.img_pitch;
                for (int k = lt; k < N; k += T) {
                    const u32 v = p.elem == 1 ? (u32)row[k] : (u32)reinterpret_cast<const u16 *>(row)[k];
                    xs[k] = make_float2((float)v, 0.f);
                }
            } else if (p.load == LOAD_COMPLEX) {
                const float2 *row = p.in + (long long)r * p.in_stride;
                for (int k = lt; k < N; k += T) xs[k] = row[k];
            } else {
                // the PSF's taps that land on grid row r, scattered onto the row's columns
                const int taps = p.kh * p.kw;
                for (int q = lt; q < taps; q += T) {
                    const int i = q / p.kw, j = q - i * p.kw;
                    int gr = (i - p.kh / 2) % p.grid_rows;
                    if (gr < 0) gr += p.grid_rows;
                    if (gr != r) continue;
                    int gc = (j - p.kw / 2) % N;
                    if (gc < 0) gc += N;
                    atomicAdd(&xs[gc].x, p.psf[q]);
                }
            }
        }
        __syncthreads();
        if (p.op == OP_FILTER) {
            dft_row(xs, p.t, ts, false, lt, T);
            // conj(P) / (|P|^2 + nsr)
            const float2 *ps = p.pspec + (long long)(live ? r : 0) * p.pspec_stride;
            for (int k = lt; k < N; k += T) {
                const float2 P = ps[k];
                const float den = P.x * P.x + P.y * P.y + p.nsr;
                xs[k] = cmul(xs[k], make_float2(P.x / den, -P.y / den));
            }
            __syncthreads();
            dft_row(xs, p.t, ts, true, lt, T);
        } else {
            dft_row(xs, p.t, ts, p.op == OP_INV, lt, T);
        }
        if (live && p.store == STORE_COMPLEX) {
            float2 *row = p.out + (long long)r * p.out_stride;
            for (int k = lt; k < N; k += T) row[k] = xs[k];
        } else if (live) {
            uint8_t *row = p.dst + (long long)r * p.dst_pitch;
            for (int k = lt; k < N; k += T) {
                const float y = xs[k].x * p.scale;
                if (p.y_out) p.y_out[(long long)r * N + k] = y;
                // floor(y + 0.5) clamped to [0, maxv]: the round-down conversion
                // saturates negatives (and NaN) to 0
                const u32 q = min(__float2uint_rd(y + 0.5f), p.maxv);
                if (p.elem == 1) row[k] = (uint8_t)q;
                else reinterpret_cast<u16 *>(row)[k] = (u16)q;
            }
        }
        __syncthreads();
    }
}

// out (C x R) = transpose of in (R x C), 32 x 32 tiles through shared memory.
__global__ void fft_transpose_kernel(const float2 *__restrict__ in, float2 *__restrict__ out, int R, int C)
{
    __shared__ float2 tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int r = by + j, c = bx + threadIdx.x;
        if (r < R && c < C) tile[j][threadIdx.x] = in[(long long)r * C + c];
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += blockDim.y) {
        const int c = bx + j, r = by + threadIdx.x;
        if (c < C && r < R) out[(long long)c * R + r] = tile[threadIdx.x][j];
    }
}

// Twiddles for M, and for Bluestein the chirp of N and the chirp filter b
// (b_m = conj(w_m) for m < N, b_{M-m} = conj(w_m) for 0 < m < N, else 0),
// in binary64 rounded to binary32.  k^2 is reduced modulo 2N exactly first.
__global__ void fft_tables_kernel(float2 *tw, int M, float2 *chirp, float2 *bbuf, int N, int bluestein)
{
    const int stride = gridDim.x * blockDim.x;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M / 2; k += stride) {
        double s, c;
        sincospi(-2.0 * (double)k / (double)M, &s, &c);
        tw[k] = make_float2((float)c, (float)s);
    }
    if (!bluestein) return;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M; k += stride) {
        const int m = k < N ? k : (k > M - N ? M - k : -1);
        float2 b = make_float2(0.f, 0.f);
        if (m >= 0) {
            const long long q = ((long long)m * (long long)m) % (2LL * N);
            double s, c;
            sincospi(-(double)q / (double)N, &s, &c);
            if (k < N) chirp[k] = make_float2((float)c, (float)s);
            b = make_float2((float)c, -(float)s);
        }
        bbuf[k] = b;
    }
}

}  // namespace

// ---------------------------------------------------------------- host side
namespace {

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

// Transform length M and log2 M of a row length N (0 if N is beyond the limits).
void len_plan(int N, int &M, int &logM)
{
    M = 0;
    logM = 0;
    if (N < 1) return;
    int m = is_pow2(N) ? N : 1;
    if (!is_pow2(N))
        while (m < 2 * N - 1) m <<= 1;
    if (m > kMaxM) return;
    M = m;
    while ((1 << logM) < M) ++logM;
}

struct FftLayout {
    int N[2], M[2], logM[2];                  // [0]: rows of W, [1]: columns of H
    size_t tw[2], chirp[2], bbuf[2], bhat[2];
    size_t A, B, P, total;
};

bool fft_layout(int H, int W, FftLayout &L)
{
    L.N[0] = W;
    L.N[1] = H;
    size_t off = 0;
    for (int d = 0; d < 2; ++d) {
        len_plan(L.N[d], L.M[d], L.logM[d]);
        if (!L.M[d]) return false;
        const size_t M = (size_t)L.M[d], N = (size_t)L.N[d];
        const bool blue = M != N;
        L.tw[d] = off;
        off += round_up(std::max<size_t>(1, M / 2) * sizeof(float2), kAlign);
        L.chirp[d] = off;
        off += blue ? round_up(N * sizeof(float2), kAlign) : 0;
        L.bbuf[d] = off;
        off += blue ? round_up(M * sizeof(float2), kAlign) : 0;
        L.bhat[d] = off;
        off += blue ? round_up(M * sizeof(float2), kAlign) : 0;
    }
    const size_t plane = round_up((size_t)H * (size_t)W * sizeof(float2), kAlign);
    L.A = off;
    L.B = L.A + plane;
    L.P = L.B + plane;
    L.total = L.P + plane;
    return true;
}

LenTables tables_of(uint8_t *ws, const FftLayout &L, int d)
{
    LenTables t;
    t.N = L.N[d];
    t.M = L.M[d];
    t.logM = L.logM[d];
    t.tw = reinterpret_cast<const float2 *>(ws + L.tw[d]);
    t.chirp = reinterpret_cast<const float2 *>(ws + L.chirp[d]);
    t.bhat = reinterpret_cast<const float2 *>(ws + L.bhat[d]);
    return t;
}

std::mutex g_attr_mu;
bool g_attr_set = false;

cudaError_t launch_rows(const RowParams &p, cudaStream_t s)
{
    {
        std::lock_guard<std::mutex> lk(g_attr_mu);
        if (!g_attr_set) {
            const cudaError_t e = cudaFuncSetAttribute(fft_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                       (int)(2 * kMaxM * sizeof(float2)));
            if (e != cudaSuccess) return e;
            g_attr_set = true;
        }
    }
    const int R = rows_per_cta(p.t.M);
    const int grid = std::min((p.rows + R - 1) / R, 65535);
    // R rows, then the per-stage twiddle table (M - 1 entries)
    const size_t smem = ((size_t)R * p.t.M + (size_t)p.t.M) * sizeof(float2);
    fft_rows_kernel<<<grid, kFftThreads, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_transpose(const float2 *in, float2 *out, int R, int C, cudaStream_t s)
{
    const dim3 block(32, 8), grid((C + 31) / 32, (R + 31) / 32);
    fft_transpose_kernel<<<grid, block, 0, s>>>(in, out, R, C);
    return cudaGetLastError();
}

RowParams row_params(const LenTables &t, int rows)
{
    RowParams p;
    std::memset(&p, 0, sizeof(p));
    p.t = t;
    p.rows = rows;
    return p;
}

// Twiddles (and the Bluestein chirp and its filter's transform) of one length.
cudaError_t setup_tables(uint8_t *ws, const FftLayout &L, int d, cudaStream_t s)
{
    const int N = L.N[d], M = L.M[d];
    const bool blue = M != N;
    float2 *tw = reinterpret_cast<float2 *>(ws + L.tw[d]);
    float2 *chirp = reinterpret_cast<float2 *>(ws + L.chirp[d]);
    float2 *bbuf = reinterpret_cast<float2 *>(ws + L.bbuf[d]);
    const int blocks = std::max(1, std::min(64, (M + 255) / 256));
    fft_tables_kernel<<<blocks, 256, 0, s>>>(tw, M, chirp, bbuf, N, blue ? 1 : 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !blue) return e;
    // bhat = DFT_M(b): the power-of-two transform of length M
    LenTables tm;
    tm.N = M;
    tm.M = M;
    tm.logM = L.logM[d];
    tm.tw = tw;
    tm.chirp = nullptr;
    tm.bhat = nullptr;
    RowParams p = row_params(tm, 1);
    p.load = LOAD_COMPLEX;
    p.in = bbuf;
    p.in_stride = M;
    p.op = OP_FWD;
    p.store = STORE_COMPLEX;
    p.out = reinterpret_cast<float2 *>(ws + L.bhat[d]);
    p.out_stride = M;
    return launch_rows(p, s);
}

}  // namespace

extern "C" {

hd_status wiener_deconv_workspace_size(int H, int W, size_t *bytes)
{
    if (!bytes || H < 1 || W < 1) return HD_ERR_ARG;
    FftLayout L;
    if (!fft_layout(H, W, L)) return HD_ERR_OVERFLOW;
    *bytes = L.total;
    return HD_OK;
}

hd_status wiener_deconvolve(const hd_image *img, const float *psf, int kh, int kw, double nsr, void *workspace,
                            size_t ws_bytes, hd_stream_t stream)
{
    if (!img) return HD_ERR_ARG;
    if (img->dtype != HD_U8 && img->dtype != HD_U16) return HD_ERR_DTYPE;
    if (img->dtype == HD_U8 && img->p.bits != 8) return HD_ERR_DTYPE;
    if (img->dtype == HD_U16 && (img->p.bits < 1 || img->p.bits > 16)) return HD_ERR_DTYPE;
    if (img->H < 1 || img->W < 1) return HD_ERR_ARG;
    FftLayout L;
    if (img->H > HD_DIM_MAX || img->W > HD_DIM_MAX || !fft_layout(img->H, img->W, L)) return HD_ERR_OVERFLOW;
    if (!img->src || !img->dst) return HD_ERR_ARG;
    const size_t es = img->dtype == HD_U8 ? 1 : 2, row = (size_t)img->W * es;
    if (img->src_pitch < row || img->dst_pitch < row) return HD_ERR_ARG;
    if (es == 2 && ((((uintptr_t)img->src | (uintptr_t)img->dst) & 1) || ((img->src_pitch | img->dst_pitch) & 1)))
        return HD_ERR_ARG;
    const uintptr_t s0 = (uintptr_t)img->src, s1 = s0 + (size_t)(img->H - 1) * img->src_pitch + row;
    const uintptr_t d0 = (uintptr_t)img->dst, d1 = d0 + (size_t)(img->H - 1) * img->dst_pitch + row;
    if (s0 < d1 && d0 < s1) return HD_ERR_ARG;
    if (!psf || ((uintptr_t)psf & 3) || kh < 1 || kw < 1 || kh > HD_PSF_MAX || kw > HD_PSF_MAX) return HD_ERR_ARG;
    if (!(nsr >= 0.0) || !std::isfinite(nsr)) return HD_ERR_ARG;
    if (img->y_out && ((uintptr_t)img->y_out & 3)) return HD_ERR_ARG;
    if (!workspace || ((uintptr_t)workspace % kAlign) || ws_bytes < L.total) return HD_ERR_WORKSPACE;

    cudaStream_t s = (cudaStream_t)stream;
    uint8_t *ws = static_cast<uint8_t *>(workspace);
    const int H = img->H, W = img->W;
    float2 *A = reinterpret_cast<float2 *>(ws + L.A);
    float2 *B = reinterpret_cast<float2 *>(ws + L.B);
    float2 *Pt = reinterpret_cast<float2 *>(ws + L.P);
    if (setup_tables(ws, L, 0, s) != cudaSuccess) return HD_ERR_CUDA;
    if (setup_tables(ws, L, 1, s) != cudaSuccess) return HD_ERR_CUDA;
    const LenTables tW = tables_of(ws, L, 0), tH = tables_of(ws, L, 1);

    // the PSF's transfer function, columns as rows: Pt (W x H)
    RowParams p = row_params(tW, H);
    p.load = LOAD_PSF;
    p.psf = psf;
    p.kh = kh;
    p.kw = kw;
    p.grid_rows = H;
    p.op = OP_FWD;
    p.store = STORE_COMPLEX;
    p.out = A;
    p.out_stride = W;
    if (launch_rows(p, s) != cudaSuccess) return HD_ERR_CUDA;
    if (launch_transpose(A, Pt, H, W, s) != cudaSuccess) return HD_ERR_CUDA;
    p = row_params(tH, W);
    p.load = LOAD_COMPLEX;
    p.in = Pt;
    p.in_stride = H;
    p.op = OP_FWD;
    p.store = STORE_COMPLEX;
    p.out = Pt;
    p.out_stride = H;
    if (launch_rows(p, s) != cudaSuccess) return HD_ERR_CUDA;

    // the image: row DFTs, columns as rows, column DFT x filter x inverse
    // column DFT, back, inverse row DFTs with the 1/(HW) scale and rounding
    p = row_params(tW, H);
    p.load = LOAD_IMAGE;
    p.img = static_cast<const uint8_t *>(img->src);
    p.img_pitch = (long long)img->src_pitch;
    p.elem = (int)es;
    p.op = OP_FWD;
    p.store = STORE_COMPLEX;
    p.out = A;
    p.out_stride = W;
    if (launch_rows(p, s) != cudaSuccess) return HD_ERR_CUDA;
    if (launch_transpose(A, B, H, W, s) != cudaSuccess) return HD_ERR_CUDA;
    p = row_params(tH, W);
    p.load = LOAD_COMPLEX;
    p.in = B;
    p.in_stride = H;
    p.op = OP_FILTER;
    p.pspec = Pt;
    p.pspec_stride = H;
    p.nsr = (float)nsr;
    p.store = STORE_COMPLEX;
    p.out = B;
    p.out_stride = H;
    if (launch_rows(p, s) != cudaSuccess) return HD_ERR_CUDA;
    if (launch_transpose(B, A, W, H, s) != cudaSuccess) return HD_ERR_CUDA;
    p = row_params(tW, H);
    p.load = LOAD_COMPLEX;
    p.in = A;
    p.in_stride = W;
    p.op = OP_INV;
    p.store = STORE_IMAGE;
    p.dst = static_cast<uint8_t *>(img->dst);
    p.dst_pitch = (long long)img->dst_pitch;
    p.elem = (int)es;
    p.scale = (float)(1.0 / ((double)H * (double)W));
    p.maxv = (u32)((1u << img->p.bits) - 1u);
    p.y_out = img->y_out;
    if (launch_rows(p, s) != cudaSuccess) return HD_ERR_CUDA;
    return HD_OK;
}

}  // extern "C"
