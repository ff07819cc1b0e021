// hd_internal.h -- types shared by the persistent kernel and the host API.
//
// Work decomposition: every image is cut into output tiles of about
// (64 - 2 Rw) x (region_h - 2 Ry) pixels, Rw = w/2 and Ry = wh/2 the Wiener
// window's column and row radii (0 for the median alone), so that tile plus
// Wiener halo is a 64 x region_h region.  A work item is
// (image, phase, tile).  Items are taken in ticket
// order from one global counter by the CTAs of a persistent grid, so a CTA
// only ever waits on items that running CTAs already hold.
#pragma once
#include <cstdint>

namespace hd {

// What an image's two phases do.
enum Mode : int {
    MODE_AMF = 0,           // P1: median -> dst
    MODE_WIENER_EST = 1,    // P1: stats of src (sum D); P2: Wiener apply src -> dst
    MODE_WIENER_GIVEN = 2,  // P1: Wiener apply src -> dst (nu2 supplied)
    MODE_HYBRID_EST = 3,    // P1: median (+ Wiener halo) + stats, median -> fbuf; P2: apply fbuf -> dst
    MODE_HYBRID_GIVEN = 4,  // P1: median (+ Wiener halo) then apply in shared memory -> dst
};

inline bool mode_two_phase(int m) { return m == MODE_WIENER_EST || m == MODE_HYBRID_EST; }
inline bool mode_has_amf(int m) { return m == MODE_AMF || m == MODE_HYBRID_EST || m == MODE_HYBRID_GIVEN; }
inline bool mode_has_wiener(int m) { return m != MODE_AMF; }

// Per-image control block in the workspace (64 bytes, zero between launches).
// sum over pixels of D = n*S2 - S1^2 is n*B - A, both exact integers:
//   A = sum over pixels p of S1_p^2,  B = sum over pixels q of M(q) f_q^2,
// M(q) = number of (pixel, window offset) pairs whose sample is q.
// Each tile adds the low and high 32-bit halves of its 64-bit partials to
// separate 64-bit words (A = A_hi32 * 2^32 + A_lo32), so the adds need no
// returned value and cannot overflow for fewer than 2^32 tiles.
struct ImgCtl {
    unsigned long long A_lo32, A_hi32;
    unsigned long long B_lo32, B_hi32;
    unsigned int p1_done;         // phase-1 tiles finished
    unsigned int pad[7];
};
static_assert(sizeof(ImgCtl) == 64, "ImgCtl layout");

struct ImgDesc {
    const uint8_t *src;
    uint8_t *dst;
    uint8_t *fbuf;            // median output plane (MODE_HYBRID_EST)
    long long src_pitch, dst_pitch, f_pitch;   // bytes
    double noise_var;
    double inv_den;           // RN(1 / (n^2 H W)), for the correctly rounded noise-variance quotient         // < 0: estimate
    double *noise_var_out;    // optional
    float *y_out;             // optional, pitch W floats
    ImgCtl *ctl;
    int H, W;
    int elem;                 // bytes per pixel: 1 or 2
    int maxv;                 // 2^bits - 1
    int smax;                 // odd >= 3 (ignored when the mode has no median)
    int w;                    // Wiener window columns, odd >= 1 (ignored when the mode has no Wiener stage)
    int wh;                   // Wiener window rows, odd >= 1
    int unresolved;           // 0: zmed of Smax window, 1: keep input
    int border_zero;          // Wiener border: 0 symmetric, 1 zero
    int mode;
    int tiles_x, tiles_y;
    int p2_items;             // phase-2 queue items: the tiles (recompute pass), 0 with the plane
    float *plane;             // optional (estimated noise variance): per output pixel the
                              // binary32 pair (mu, s2) left by phase 1, row-major, W pairs a row;
                              // nullptr: phase 2 recomputes the sums from the f region
    // A part of a larger image (one image split by row strips): the buffers
    // hold rows [gy_off, gy_off + H) of an image of Hg rows, and the part owns
    // (tiles, statistics and output) local rows [own0, own1).  A whole image:
    // Hg = H, gy_off = 0, own0 = 0, own1 = H.
    int Hg, gy_off, own0, own1;
};

// A run of consecutive tickets belonging to one (image, phase).
struct Seg {
    int img;
    int phase;        // 1 or 2
    int first;        // first ticket
    int count;        // number of tiles
};

// Kernel parameters.  Single-image launches carry the descriptor inline;
// batched launches point at tables in the workspace.
struct LaunchParams {
    const ImgDesc *descs;     // device table, or nullptr -> use one
    const Seg *segs;          // device table, or nullptr -> use oneseg
    ImgDesc one;
    Seg oneseg[2];
    int nsegs;
    int total_items;
    unsigned int *ticket;     // device counters {ticket, exited CTAs}; zero before the first launch,
                              // reset to zero by the last CTA to exit
    ImgCtl *ctl_reset;        // control blocks the last CTA zeroes (nctl of them)
    int nctl;
    int region_h;             // rows of the f region: multiple of 8 in [16, 128]
    int ra_max;               // largest median halo over the launch (shared memory sizing)
    int wide;                 // some image needs 64-bit Wiener sums
    unsigned long long spin_limit;   // bounded wait, in polls
    int p2_plane;             // 1: `one` has a statistics plane; after the queue every CTA applies
                              // its own 1/gridDim share of the image's pixels from it
    int p2_direct;            // with the plane: 1 reads it straight from L2 (the phase-2 working set
                              // fits the L2), 0 stages it through shared memory by bulk copies
    int small_growth;         // growth by one warp without barriers when at most this many pixels
                              // of a region fail level A at 3x3 (0: never)
    int select_lanes;         // cap on the lanes sharing one median selection (0: per window size)
};

// Shared-memory bytes the kernel needs.
size_t smem_bytes(int region_h, int ra_max, int wide);

// Upload `bytes` of a host table to device memory with parameter-carrying
// kernel launches on `stream` (asynchronous, capturable); returns cudaError_t.
constexpr int kTableChunkBytes = 30 * 1024;
int launch_table_upload(void *dst, const void *src, size_t bytes, void *stream);

// Launch the persistent kernel; returns cudaError_t as int.
int launch_persistent(const LaunchParams &lp, int grid, size_t smem, void *stream);

// Largest CTAs per SM for a shared-memory size (occupancy), and the SM count.
int max_ctas_per_sm(size_t smem);
int sm_count();

// Device error word helpers.
int read_and_clear_device_error(unsigned int *out);

// The argument checks of hybrid_denoise, in its order; returns an hd_status value.
int check_hybrid_image(const void *img);

// hybrid_denoise on a caller-provided workspace (used by the entry point whose
// scratch is a static device array); returns an hd_status value.
int hybrid_on_workspace(const void *img, void *ws, size_t ws_bytes, void *stream);

// Bytes at the start of a hybrid workspace that must be zero before a launch.
size_t hybrid_control_bytes();
// Smallest workspace that hybrid_on_workspace accepts for the image (no plane).
size_t hybrid_min_bytes(const void *img);

constexpr int kThreads = 256;
// With the statistics plane, phase 2 streams each CTA's share of the pixels
// (row-major order) in units of up to kUnitPx, staged in shared memory by
// bulk copies up to kStages units ahead; every thread applies four pixels of
// a unit.
constexpr int kUnitPx = kThreads * 4;
constexpr int kStages = 4;
constexpr unsigned int DEVERR_TIMEOUT = 1u;

}  // namespace hd
