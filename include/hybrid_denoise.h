/*
 * hybrid_denoise.h -- C ABI of the GB300 hybrid multi-noise denoiser.
 *
 * Method: Youssef, Mahmoud, El-Horbaty, "A Parallel Hybrid Technique for
 * Multi-Noise Removal from Grayscale Medical Images".  The hybrid is an
 * adaptive median filter (Algorithm 1, step 6; Section IV) followed by a
 * Wiener filter (Algorithm 1, step 4d), here in its spatial local-statistics
 * form with the noise variance estimated as the mean local variance.
 *
 * Conventions for every entry point
 *   - Images are H x W, row-major, with a row pitch in BYTES (>= W * element
 *     size).  HD_U8 images hold 8-bit values; HD_U16 images hold values of
 *     `bits` bits (1..16; values above 2^bits - 1 are outside the contract).
 *   - src, dst, workspace and every optional output are DEVICE pointers owned
 *     by the caller (hybrid_denoise_host is the one exception: src and dst are
 *     host pointers there).  The library allocates no device memory.
 *   - src and dst must not overlap: the adaptive median reads only the noisy
 *     input (the listing's neighbourhood statistics are taken of g, never of
 *     the partly filtered copy).  contrast_stretch alone also runs in place.
 *   - Work is enqueued on `stream` (NULL = legacy default stream).  Argument
 *     errors are returned synchronously before anything is enqueued.  Launch
 *     failures return HD_ERR_CUDA.  Faults seen by the kernels while running
 *     (a bounded wait that ran out) are latched in a per-device error word and
 *     reported by hd_get_device_error.
 *   - A workspace must be zero-filled before its first use (cudaMemset); every
 *     call leaves the queue counters in it zeroed again for the next call.
 *     A call that did not run to completion (launch error, abort) leaves it in
 *     an unknown state: zero it again.
 *   - Calls that share a workspace must not overlap in time on the device.
 *   - No C++ exception crosses this boundary.
 */
#ifndef HYBRID_DENOISE_H
#define HYBRID_DENOISE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t. */
typedef struct CUstream_st *hd_stream_t;

typedef enum {
    HD_OK = 0,
    HD_ERR_ARG = 1,        /* null pointer, bad size, bad pitch, overlap, bad enum */
    HD_ERR_SMAX = 2,       /* Smax not an odd integer in [3, HD_SMAX_MAX] (Alg. 1, step 6a) */
    HD_ERR_WINDOW = 3,     /* Wiener window side not odd in [1, HD_WIENER_W_MAX] */
    HD_ERR_DTYPE = 4,      /* unknown dtype or bits outside 1..16 (8 for HD_U8) */
    HD_ERR_WORKSPACE = 5,  /* workspace missing, misaligned or smaller than required */
    HD_ERR_CUDA = 6,       /* a CUDA runtime call failed */
    HD_ERR_TIMEOUT = 7,    /* a bounded device-side wait ran out (hd_get_device_error) */
    HD_ERR_OVERFLOW = 8    /* size beyond the library's limits */
} hd_status;

typedef enum { HD_U8 = 0, HD_U16 = 1 } hd_dtype;

/* Border rule for out-of-image window samples.  SYMMETRIC: half-sample
 * reflection with period 2N (... 1 0 | 0 1 ... N-1 | N-1 N-2 ...), used by both
 * stages.  ZERO: samples outside the image read 0 but still count in the
 * window size n = w*w; Wiener stage only. */
typedef enum { HD_BORDER_SYMMETRIC = 0, HD_BORDER_ZERO = 1 } hd_border;

/* Pixels that fail level A for every window up to Smax.  ZMED: they take the
 * median of the Smax window (textbook adaptive median; replaces isolated
 * impulses on flat backgrounds).  KEEP: they keep their input value (literal
 * reading of Algorithm 1, where the working copy starts as the input). */
typedef enum { HD_UNRESOLVED_ZMED = 0, HD_UNRESOLVED_KEEP = 1 } hd_unresolved;

#define HD_SMAX_MAX 15
#define HD_WIENER_W_MAX 15
#define HD_DIM_MAX 65535          /* largest H or W */

/* Filter parameters (Algorithm 1: Smax = 11 in the paper's runs). */
typedef struct {
    int smax;            /* adaptive median: largest window, odd, 3..HD_SMAX_MAX */
    int wiener_w;        /* Wiener window side, odd, 1..HD_WIENER_W_MAX */
    double noise_var;    /* Wiener noise variance nu2 (in squared LSB); < 0: estimate it
                            as the mean over all pixels of the local variance */
    int border;          /* hd_border, Wiener stage (the median always reflects) */
    int unresolved;      /* hd_unresolved */
    int bits;            /* significant bits: 8 for HD_U8; 1..16 for HD_U16 */
    int wiener_h;        /* Wiener window rows, odd, 1..HD_WIENER_W_MAX; 0 = wiener_w
                            (square window).  The paper gives no window size. */
} hd_params;

/* One image and where its result goes. */
typedef struct {
    const void *src;         /* device, H rows of src_pitch bytes */
    void *dst;               /* device, H rows of dst_pitch bytes, same dtype */
    int H, W;                /* 1..HD_DIM_MAX each */
    size_t src_pitch;        /* bytes, >= W * element size */
    size_t dst_pitch;        /* bytes, >= W * element size */
    int dtype;               /* hd_dtype */
    hd_params p;
    double *noise_var_out;   /* optional device pointer: receives the nu2 that was used */
    float *y_out;            /* optional device pointer: H x W float plane (pitch W*4) of
                                the unrounded Wiener output */
} hd_image;

/* ---------------------------------------------------------------- stages
 * Adaptive median filter (Algorithm 1, step 6): for k = 3, 5, ..., Smax over
 * the k x k window of src, level A (zmin < zmed < zmax, strict) decides
 * whether the pixel is processed at k; level B (zmin < zxy < zmax, strict)
 * keeps zxy, else outputs zmed.  The first k that passes level A wins.
 * Output is exact (integer order statistics).  Needs no workspace.
 * Uses img->p.smax and img->p.unresolved; the Wiener fields are ignored. */
hd_status amf_filter(const hd_image *img, hd_stream_t stream);

/* Wiener filter of an already median-filtered image (Algorithm 1, step 4d;
 * local-statistics form).  Over the window of h = wiener_h rows (wiener_w when
 * 0) by w = wiener_w columns, n = h*w, with exact integer
 * S1 = sum f, S2 = sum f^2 and D = n*S2 - S1^2:
 *   mu = S1/n, sigma2 = D/n^2,
 *   nu2 = noise_var if >= 0, else fl(fl(sum of D over all pixels) / (n^2 H W)),
 *   y = mu + max(sigma2 - nu2, 0) / max(sigma2, nu2) * (f - mu)  (y = mu if both 0),
 *   dst = min(2^bits - 1, floor(y + 0.5)).
 * The sums are exact integers, nu2 is binary64, the gain and y are binary32
 * with a fixed evaluation order (documented with the kernel).
 * workspace: device, >= wiener_workspace_size() bytes, 256-byte aligned
 * (the size includes a plane of 8 bytes per pixel for the binary32 mu and
 * sigma2; a workspace without that room, down to the size returned for the
 * same image with the plane left out, is accepted and recomputes the window
 * sums in the second pass instead: same output, slower). */
hd_status wiener_filter(const hd_image *img, void *workspace, size_t ws_bytes,
                        hd_stream_t stream);
hd_status wiener_workspace_size(int H, int W, int dtype, const hd_params *p, size_t *bytes);

/* The hybrid (Algorithm 1, step 4, without the contrast stretch of step 4e,
 * which is contrast_stretch below):
 * dst = Wiener(AdaptiveMedian(src)).  One persistent kernel launch: the
 * median output stays in the workspace (L2-resident for images up to tens of
 * MB); with a caller-supplied noise_var >= 0 the whole hybrid is one pass and
 * needs no workspace.  Exactly one kernel is enqueued per call.
 * workspace: device, 256-byte aligned, >= hybrid_min_workspace_size() bytes.
 *   hybrid_workspace_size() (the median plane, the queue counters and a plane
 *   of 8 bytes per pixel holding the binary32 local mean and variance) gives
 *   the fastest path: the Wiener pass then streams those statistics instead
 *   of recomputing the window sums.  hybrid_min_workspace_size() (no
 *   statistics plane) is the least accepted; any size in between runs the
 *   recompute path.  The output is bit-identical either way. */
hd_status hybrid_denoise(const hd_image *img, void *workspace, size_t ws_bytes,
                         hd_stream_t stream);
hd_status hybrid_workspace_size(int H, int W, int dtype, const hd_params *p, size_t *bytes);
hd_status hybrid_min_workspace_size(int H, int W, int dtype, const hd_params *p, size_t *bytes);

/* A host pipeline: many images of one size and one parameter set, from host
 * buffers to host buffers, with the copies of each step overlapping the
 * kernels of the steps before and after it.  Each step is the hybrid of
 * Algorithm 1, step 4; the pipelining has no counterpart in the paper (its
 * images are single files on one CPU).  It holds `depth` slots of device
 * images (noisy in, result out) in the caller's workspace and three CUDA
 * streams of its own (copies in, kernels, copies out); step i uses slot
 * i mod depth, and events make a slot wait for its previous step.
 *   depth: 1..HD_PIPELINE_DEPTH_MAX (2 overlaps one step's copies with its
 *          neighbours' kernels).
 *   workspace: device, 256-byte aligned, >= hd_host_pipeline_workspace_size(),
 *          zero-filled before first use; owned by the caller, must outlive the
 *          pipeline.
 *   submit: src and dst are HOST pointers with row pitches in bytes (pinned
 *          memory for overlap; pageable memory works without it).  The call
 *          only enqueues: src must stay unchanged and dst unread until
 *          hd_host_pipeline_wait returns.  Same filtering, parameters and
 *          output as hybrid_denoise.
 *   wait: blocks until every submitted step has finished; HD_ERR_CUDA if a
 *          stream failed (device-side timeouts: hd_get_device_error).
 *   destroy: waits, then frees the streams and events (not the workspace).
 * One pipeline is used by one host thread at a time (its calls are not
 * synchronised with each other); separate pipelines are independent. */
#define HD_PIPELINE_DEPTH_MAX 8
typedef struct hd_host_pipeline hd_host_pipeline;
hd_status hd_host_pipeline_workspace_size(int H, int W, int dtype, const hd_params *p, int depth,
                                          size_t *bytes);
hd_status hd_host_pipeline_create(int H, int W, int dtype, const hd_params *p, int depth,
                                  void *workspace, size_t ws_bytes, hd_host_pipeline **pipeline);
hd_status hd_host_pipeline_submit(hd_host_pipeline *pipeline, const void *src, size_t src_pitch,
                                  void *dst, size_t dst_pitch);
hd_status hd_host_pipeline_wait(hd_host_pipeline *pipeline);
hd_status hd_host_pipeline_destroy(hd_host_pipeline *pipeline);

/* The hybrid with the paper's partitioned median (Algorithm 1, step 6: the
 * adaptive median of the image in `parts` sub-images, each filtered by its
 * own worker).  The image is cut into `parts` row
 * strips, strip i covering rows floor(i H / parts) .. floor((i+1) H / parts) - 1,
 * and each strip is median-filtered as an image of its own: its windows
 * reflect at the strip's edges, so pixels within Smax/2 rows of a seam can
 * differ from hybrid_denoise.  The Wiener filter then runs on the whole
 * reassembled median image.  parts = 1 is exactly hybrid_denoise.
 *   parts: 1..H, else HD_ERR_ARG.  Each strip costs one descriptor (about
 *   150 bytes) written into the workspace by small launches of 30 KB each.
 *   workspace: device, 256-byte aligned, >= hybrid_strips_workspace_size()
 *   bytes.  Each call clears the counters it uses first (a memset on the
 *   stream), so one workspace serves calls of any size and partition in turn.
 * Two persistent launches (all strips' medians in one, then the Wiener), plus
 * the memset and one small launch that writes the strip descriptors into the
 * workspace (parts = 1: the memset and hybrid_denoise's single launch). */
hd_status hybrid_denoise_strips(const hd_image *img, int parts, void *workspace, size_t ws_bytes,
                                hd_stream_t stream);
hd_status hybrid_strips_workspace_size(int H, int W, int dtype, const hd_params *p, int parts,
                                       size_t *bytes);

/* The hybrid over host buffers: img->src and img->dst are HOST pointers
 * (pinned memory gives overlap-free full-speed copies; pageable works).  The
 * call copies src into the workspace, runs hybrid_denoise there, copies the
 * result back to dst and waits for the stream.  Returns after dst is written.
 * A host buffer whose pitch equals W * element size moves as one linear copy;
 * a padded one moves row by row (slower for many short rows).
 * workspace: device, >= hybrid_host_workspace_size() bytes. */
hd_status hybrid_denoise_host(const hd_image *img, void *workspace, size_t ws_bytes,
                              hd_stream_t stream);
hd_status hybrid_host_workspace_size(int H, int W, int dtype, const hd_params *p,
                                     size_t *bytes);

/* The hybrid with no device allocation anywhere: the scratch (median plane
 * and queue counters) is one array of HD_STATIC_SCRATCH_BYTES in device
 * memory that the library declares, so a caller that cannot call cudaMalloc
 * (a fixed-budget real-time loop, a plug-in whose host owns the allocator)
 * can still run the hybrid on its own src/dst buffers.  The paper has no
 * counterpart; this is a deployment convenience.
 *   - Limit: images whose hybrid_min_workspace_size() exceeds
 *     HD_STATIC_SCRATCH_BYTES (36 MiB: e.g. 4096 x 4096 at 16 bits fits, and
 *     1620 x 1620 at 8 bits) are rejected with HD_ERR_OVERFLOW.  Images whose
 *     hybrid_workspace_size() also fits take the statistics-plane path.
 *   - Every GPU that loads the library holds the array until the process
 *     exits.
 *   - The first call on each device looks up the array's device address
 *     (with that device current), and so does the first call after the
 *     device's context was destroyed and created again (cudaDeviceReset);
 *     make those calls before any stream capture.
 *   - All calls on a device share the one array: calls that overlap in time
 *     on the GPU race and corrupt each other's results.  The array keeps the
 *     last call's contents; each call clears the queue counters it needs.
 * Same filtering, parameters and output as hybrid_denoise, and the same
 * argument errors in the same order; HD_ERR_OVERFLOW for a size beyond the
 * array comes after them. */
#define HD_STATIC_SCRATCH_BYTES (36u * 1024u * 1024u)
hd_status hybrid_denoise_static(const hd_image *img, hd_stream_t stream);

/* ---------------------------------------------------------------- image parts
 * One image split across GPUs by row strips, one part per GPU: the paper's
 * partitioned parallel step (Algorithm 1, step 6, parfor over the image's
 * sub-images; Fig. 5), here with whole-image results.  Each part computes
 * the output rows it owns exactly as hybrid_denoise does for the whole image:
 * it holds its own rows plus the halo rows that their windows read (copied
 * from the neighbouring parts first), and the one image-wide quantity, the
 * noise variance (mean local variance, Algorithm 1, step 4d), comes from four
 * exact integer sums that the caller adds over all parts between the two
 * calls (an all-reduce).  The reassembled image is bit-identical to
 * hybrid_denoise of the whole image.
 *   H, W:     the WHOLE image.
 *   buf_row0, buf_rows: the rows src holds, [buf_row0, buf_row0 + buf_rows).
 *             They must include [max(0, own_row0 - h), min(H, own_row0 +
 *             own_rows + h)), h = hd_part_halo_rows() = smax/2 + (window rows)/2.
 *   own_row0, own_rows: the rows this part owns and writes.
 *   src:      device, buf_rows rows of src_pitch bytes (the noisy image).
 *   dst:      device, own_rows rows of dst_pitch bytes: dst row 0 is image
 *             row own_row0.  Must not overlap src (hybrid_part_apply).
 *   p:        as for hybrid_denoise; noise_var must be < 0 (estimated: with a
 *             known noise variance there is nothing to exchange; run
 *             hybrid_denoise on each part's buffer and keep its own rows).
 * hybrid_part_stats: the median and the local statistics of the own rows
 *   (one persistent launch); writes the part's four sums to sums_out
 *   (device, 8-byte aligned, 4 x uint64: the low and high 32-bit halves of
 *   A = sum S1^2 and of B = sum M(q) f^2, accumulated in 64-bit words).
 * The caller adds the four words over all parts, word by word (uint64 or
 *   int64 sum; exact for fewer than 2^32 tiles in all), e.g. with one NCCL
 *   all-reduce, and passes the result to
 * hybrid_part_apply: the Wiener output of the own rows into dst (one
 *   persistent launch), with nu2 from the summed words.
 * workspace: device, 256-byte aligned, >= hybrid_part_workspace_size(); the
 *   same workspace for both calls of a part (the median and statistics planes
 *   live in it between them).  hybrid_part_stats clears what it needs. */
typedef struct {
    const void *src;
    size_t src_pitch;
    void *dst;
    size_t dst_pitch;
    int H, W;
    int buf_row0, buf_rows;
    int own_row0, own_rows;
    int dtype;
    hd_params p;
} hd_part;
hd_status hd_part_halo_rows(const hd_params *p, int *rows);
hd_status hybrid_part_workspace_size(const hd_part *part, size_t *bytes);
hd_status hybrid_part_stats(const hd_part *part, void *workspace, size_t ws_bytes, unsigned long long *sums_out,
                            hd_stream_t stream);
hd_status hybrid_part_apply(const hd_part *part, const unsigned long long *sums, void *workspace, size_t ws_bytes,
                            hd_stream_t stream);

/* ---------------------------------------------------------------- reference
 * Noise variance of an image against a clean reference (Algorithm 1, step 4d
 * hands the original image to the Wiener stage; this reads it as the source
 * of the noise variance):
 *   nu2 = fl64(fl64(S) / (H W)),  S = sum over pixels of (f - ref)^2, exact.
 * Pass the result as hd_params.noise_var: the hybrid is then one fused pass.
 *   f, ref: device images, H x W, row pitches in bytes (>= W * element size),
 *           same dtype; they may overlap (both are only read).
 *   nu2_out: device pointer, 8-byte aligned; written when the launch ends.
 *   workspace: device, 256-byte aligned, >= HD_REFNOISE_WORKSPACE_BYTES,
 *           zero-filled before first use; each call leaves it zeroed.
 * One kernel launch; no device-side waits. */
#define HD_REFNOISE_WORKSPACE_BYTES 256u
hd_status reference_noise_variance(const void *f, size_t f_pitch, const void *ref, size_t ref_pitch, int H,
                                   int W, int dtype, double *nu2_out, void *workspace, size_t ws_bytes,
                                   hd_stream_t stream);

/* ---------------------------------------------------------------- Fourier domain
 * The Wiener filter in the Fourier domain, where Section IV places the
 * hybrid's Wiener stage: deconvolution by a point-spread function with a
 * noise-to-signal ratio (the paper gives neither; both are the caller's).
 * With G the 2-D DFT of src and P the PSF's transfer function (the PSF placed
 * on the H x W grid with its centre tap, row kh/2 and column kw/2, at the
 * origin and the other taps wrapped around),
 *   F = conj(P) / (|P|^2 + nsr) * G,   y = Re IDFT(F),
 *   dst = min(2^bits - 1, max(0, floor(y + 1/2))),
 * with the DFT's periodic extension as the border rule (circular boundary).
 * Arithmetic: binary32 transforms (radix 2, and Bluestein's method for other
 * lengths) with twiddles rounded from binary64; tests bound |y - y64|.
 *   img: src, dst device images (H x W, same dtype; no overlap), p.bits;
 *        y_out optional (binary32 y, pitch W floats); the other fields are
 *        ignored.  H and W: powers of two up to 8192, or any length up to
 *        4096; else HD_ERR_OVERFLOW.
 *   psf: device, kh x kw binary32, row-major, 1 <= kh, kw <= HD_PSF_MAX.
 *   nsr: >= 0 and finite (nsr = 0 with a PSF whose transfer function
 *        vanishes somewhere divides by zero, as the formula does).
 *   workspace: device, 256-byte aligned, >= wiener_deconv_workspace_size()
 *        (three H x W complex planes and the transform tables).
 * Ten kernel launches, no device-side waits. */
#define HD_PSF_MAX 255
hd_status wiener_deconv_workspace_size(int H, int W, size_t *bytes);
hd_status wiener_deconvolve(const hd_image *img, const float *psf, int kh, int kw, double nsr, void *workspace,
                            size_t ws_bytes, hd_stream_t stream);

/* ---------------------------------------------------------------- contrast
 * Contrast stretch, the post-processing step of the hybrid (Algorithm 1,
 * step 4e).  The paper gives no rule; this is a linear stretch between two
 * saturation limits taken from the image histogram, with at most k pixels
 * saturating at each end:
 *   k  = floor(fl64(tol * N)), N = H * W, 0 <= tol < 0.5 (tol = 0: min-max),
 *   lo = the k-th smallest pixel value (counting from 0), hi = the k-th largest,
 *   dst = src where lo == hi, else
 *   dst = floor((clamp(src, lo, hi) - lo) * maxv / (hi - lo) + 1/2),
 * maxv = 2^bits - 1, in exact integer arithmetic (round half up).  Values
 * above maxv are outside the contract (they count as maxv).
 *   img: src and dst device images of the same size and dtype; dst == src with
 *        the same pitch runs in place; any other overlap is HD_ERR_ARG.  Only
 *        img->p.bits is used; noise_var_out and y_out are ignored.
 *   tol: outside [0, 0.5) or NaN is HD_ERR_ARG.
 *   workspace: device, 256-byte aligned, >= contrast_workspace_size() bytes
 *        (a 256-byte control block and a 2^bits-entry histogram), zero-filled
 *        before first use; each call leaves it zeroed.
 * One kernel launch.  Its CTAs wait for one another (bounded): a wait that
 * runs out (e.g. when other work holds the GPU's SMs so long that the grid is
 * not resident at once) latches HD_ERR_TIMEOUT for hd_get_device_error and
 * leaves dst unwritten. */
hd_status contrast_stretch(const hd_image *img, double tol, void *workspace, size_t ws_bytes,
                           hd_stream_t stream);
hd_status contrast_workspace_size(int H, int W, int dtype, const hd_params *p, size_t *bytes);

/* ---------------------------------------------------------------- batches
 * Many images of uneven sizes and per-image parameters (each the hybrid of
 * Algorithm 1, step 4; the paper runs one image at a time) in ONE persistent
 * kernel launch: a device work queue of (image, phase, tile) items where an
 * image's Wiener tiles start as soon as that image's median tiles are done,
 * so one image's Wiener overlaps another's median.  Each result is
 * bit-identical to the same image through hybrid_denoise (integer
 * reductions make the order irrelevant).
 * A batch uses the recompute Wiener pass (no statistics plane): each image's
 * Wiener tiles already run beside the next image's median tiles.
 * hybrid_denoise_batched writes the n descriptors into the workspace with
 * small kernels on `stream` (their bytes travel as kernel parameters), so the
 * call never waits for the device; the host array may be freed on return. */
hd_status hybrid_denoise_batched(const hd_image *imgs, int n, void *workspace,
                                 size_t ws_bytes, hd_stream_t stream);
hd_status hybrid_batched_workspace_size(const hd_image *imgs, int n, size_t *bytes);

/* A batch plan fixes the descriptors once (synchronous copy into the
 * workspace at creation) and replays the batch as a CUDA graph (memset of the
 * queue counters + the persistent kernel).  The plan holds host memory only;
 * the workspace stays owned by the caller and must outlive the plan. */
typedef struct hd_batch_plan hd_batch_plan;
hd_status hd_batch_plan_create(const hd_image *imgs, int n, void *workspace, size_t ws_bytes,
                               hd_batch_plan **plan);
hd_status hd_batch_plan_launch(hd_batch_plan *plan, hd_stream_t stream);
hd_status hd_batch_plan_destroy(hd_batch_plan *plan);

/* A batch pipeline: the same batch (sizes, dtypes and parameters fixed at
 * creation) run again and again from host buffers to host buffers, each step
 * the batched hybrid above (Algorithm 1, step 4 for every image; the
 * pipelining has no counterpart in the paper).  It holds `depth` slots, each
 * with device planes for every image (noisy in, result out, tight rows) and a
 * batch plan over them, and three CUDA streams of its own (copies in, kernels,
 * copies out); step i uses slot i mod depth and events make a slot wait for
 * its previous step, so one step's copies overlap its neighbours' kernels.
 *   imgs, n: the batch; only H, W, dtype and p of each image are used (src,
 *          dst, noise_var_out and y_out are ignored and may be null).
 *   depth: 1..HD_PIPELINE_DEPTH_MAX.
 *   workspace: device, 256-byte aligned, >= hd_batch_pipeline_workspace_size(),
 *          owned by the caller, must outlive the pipeline.  Creation writes the
 *          plans' tables into it (synchronous copies).
 *   submit: srcs[i] / dsts[i] are HOST pointers to image i with row pitches in
 *          bytes (pinned memory for overlap).  Images whose rows are tight and
 *          that follow each other in host memory, as they do in the slot,
 *          move as one copy.  The call only enqueues: srcs must stay unchanged
 *          and dsts unread until hd_batch_pipeline_wait returns.
 *   wait: blocks until every submitted step has finished; HD_ERR_CUDA if a
 *          stream failed (device-side timeouts: hd_get_device_error).
 *   destroy: waits, then frees the plans, streams and events.
 * One pipeline is used by one host thread at a time. */
typedef struct hd_batch_pipeline hd_batch_pipeline;
hd_status hd_batch_pipeline_workspace_size(const hd_image *imgs, int n, int depth, size_t *bytes);
hd_status hd_batch_pipeline_create(const hd_image *imgs, int n, int depth, void *workspace, size_t ws_bytes,
                                   hd_batch_pipeline **pipeline);
hd_status hd_batch_pipeline_submit(hd_batch_pipeline *pipeline, const void *const *srcs,
                                   const size_t *src_pitches, void *const *dsts, const size_t *dst_pitches);
hd_status hd_batch_pipeline_wait(hd_batch_pipeline *pipeline);
hd_status hd_batch_pipeline_destroy(hd_batch_pipeline *pipeline);

/* ---------------------------------------------------------------- tuning
 * Work-item shape and scheduling of the persistent kernel; the autotuner
 * (paper_2005_05371_gb300/autotune.py) picks them per workload class.  Each
 * item covers a region of 64 columns x region_h rows of the median output;
 * its output tile is that region less the Wiener halo,
 * (64 - 2*(w/2)) x (region_h - 2*(w/2)).  The 64 columns are fixed: each of
 * a warp's 32 lanes owns one pixel pair of a region row.
 *   region_h:     multiple of 8 in [16, 128] (default 32).
 *   ctas_per_sm:  grid size per SM, 1..8, 0 = as many as fit.
 *   plane:        0 = a single image uses the statistics plane whenever its
 *                 workspace has room for it, its Wiener pass reading the
 *                 plane straight from L2 when the plane, the median output
 *                 and the output of the image fit in the L2, else
 *                 staging it in shared memory by bulk copies; 1 = never
 *                 (recompute pass); 2 = the plane, always staged; 3 = the
 *                 plane, always read straight from L2.
 *   small_growth: when at most this many pixels of a region fail level A at
 *                 3x3, one warp grows their windows with no block barriers:
 *                 0 = default (32), -1 = never, 1..32.
 *   select_lanes: lanes that share one median selection for windows of 7x7
 *                 and more (they split the window's rows): 0 = default (up to
 *                 4 at 7x7, 8 from 9x9), or 1, 2, 4, 8 as the cap.
 *   batch_lag:    batches queue an image's Wiener tiles this many grids of
 *                 tickets after its last median tile: 0 = default (6), 1..64.
 *   batch_order:  0 = batches run in the caller's order (default); 1 = the
 *                 largest images first.
 * Applies to later launches in this process; results do not depend on it. */
typedef struct {
    int region_h;
    int ctas_per_sm;
    int plane;
    int small_growth;
    int select_lanes;
    int batch_lag;
    int batch_order;
} hd_tuning;
hd_status hd_set_tuning(const hd_tuning *t);
hd_status hd_get_tuning(hd_tuning *t);

/* Number of polls (>= 256 ns apart after the first 64) before a device-side
 * wait of a Wiener tile on its image's median tiles gives up, latches
 * HD_ERR_TIMEOUT and skips the tile.  0 restores the default (about 2 s).
 * A tiny limit makes waits run out on purpose, which is how the error path
 * is tested without stalling a GPU. */
hd_status hd_set_spin_limit(unsigned long long polls);

/* ---------------------------------------------------------------- errors
 * Synchronises `stream`, then returns and clears the device error word of the
 * current device: HD_ERR_TIMEOUT if a bounded wait inside a kernel ran out,
 * HD_ERR_CUDA if the stream reports an error, else HD_OK. */
hd_status hd_get_device_error(hd_stream_t stream);
const char *hd_status_str(hd_status s);

/* Library version as major*10000 + minor*100 + patch. */
int hd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HYBRID_DENOISE_H */
