// hd_internal.h -- types shared by the persistent kernel and the host API.
//
// Work decomposition: every image is cut into output tiles of tile_w x tile_h
// pixels.  A work item is (image, phase, tile).  Items are taken in ticket
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

// Per-image control block in the workspace (32 bytes, zeroed before a launch).
struct ImgCtl {
    unsigned long long sumD_lo;   // sum over pixels of D = n*S2 - S1^2, low word
    unsigned long long sumD_hi;   // carry word
    unsigned int p1_done;         // phase-1 tiles finished
    unsigned int pad[3];
};
static_assert(sizeof(ImgCtl) == 32, "ImgCtl layout");

struct ImgDesc {
    const uint8_t *src;
    uint8_t *dst;
    uint8_t *fbuf;            // median output plane (MODE_HYBRID_EST)
    long long src_pitch, dst_pitch, f_pitch;   // bytes
    double noise_var;         // < 0: estimate
    double *noise_var_out;    // optional
    float *y_out;             // optional, pitch W floats
    ImgCtl *ctl;
    int H, W;
    int elem;                 // bytes per pixel: 1 or 2
    int maxv;                 // 2^bits - 1
    int smax;                 // odd >= 3 (ignored when the mode has no median)
    int w;                    // odd >= 1 (ignored when the mode has no Wiener stage)
    int unresolved;           // 0: zmed of Smax window, 1: keep input
    int border_zero;          // Wiener border: 0 symmetric, 1 zero
    int mode;
    int tiles_x, tiles_y;
    int pad;
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
    int tile_w, tile_h;
    int ra_max, rw_max;       // largest halos over the launch (shared memory sizing)
    unsigned long long spin_limit;   // bounded wait, in polls
};

// Shared-memory bytes the kernel needs for a given tile and halos.
size_t smem_bytes(int tile_w, int tile_h, int ra_max, int rw_max);

// Launch the persistent kernel; returns cudaError_t as int.
int launch_persistent(const LaunchParams &lp, int grid, size_t smem, void *stream);

// Largest CTAs per SM for a shared-memory size (occupancy), and the SM count.
int max_ctas_per_sm(size_t smem);
int sm_count();

// Device error word helpers.
int read_and_clear_device_error(unsigned int *out);

constexpr int kThreads = 256;
constexpr unsigned int DEVERR_TIMEOUT = 1u;

}  // namespace hd
