// hd_api.cu -- host side of the C ABI declared in include/hybrid_denoise.h.
//
// Validates arguments, lays out the caller's workspace, builds the work-item
// segments and launches the persistent kernel (hd_kernel.cu).  No device
// memory is allocated here: every buffer comes from the caller.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "hd_contrast.h"
#include "hd_internal.h"
#include "hybrid_denoise.h"

using namespace hd;

namespace {

constexpr size_t kAlign = 256;
constexpr size_t kTicketBytes = 256;
constexpr unsigned long long kSpinLimit = 8000000ull;   // polls of >= 256 ns: about 2 s

inline size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

std::mutex g_tune_mu;
hd_tuning g_tune = {32, 0, 0, 0, 0, 0, 0};
unsigned long long g_spin_limit = kSpinLimit;

}  // namespace

unsigned long long hd::spin_limit_polls()
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return g_spin_limit;
}

namespace {

hd_tuning current_tuning()
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return g_tune;
}

int elem_size(int dtype) { return dtype == HD_U8 ? 1 : 2; }

// Rows of the Wiener window: wiener_h, or wiener_w when it is 0 (square).
int window_rows(const hd_params &p) { return p.wiener_h ? p.wiener_h : p.wiener_w; }

// Checks shared by every entry point.  `need_amf` / `need_wiener` select the
// parameter checks of the stages the call runs.
hd_status check_image(const hd_image *img, bool need_amf, bool need_wiener, bool host_buffers)
{
    if (!img) return HD_ERR_ARG;
    if (img->dtype != HD_U8 && img->dtype != HD_U16) return HD_ERR_DTYPE;
    if (img->dtype == HD_U8 && img->p.bits != 8) return HD_ERR_DTYPE;
    if (img->dtype == HD_U16 && (img->p.bits < 1 || img->p.bits > 16)) return HD_ERR_DTYPE;
    if (img->H < 1 || img->W < 1) return HD_ERR_ARG;
    if (img->H > HD_DIM_MAX || img->W > HD_DIM_MAX) return HD_ERR_OVERFLOW;
    if (!img->src || !img->dst) return HD_ERR_ARG;
    const size_t es = (size_t)elem_size(img->dtype);
    const size_t row = (size_t)img->W * es;
    if (img->src_pitch < row || img->dst_pitch < row) return HD_ERR_ARG;
    if (es == 2) {
        if ((img->src_pitch | img->dst_pitch) & 1) return HD_ERR_ARG;
        if (((uintptr_t)img->src | (uintptr_t)img->dst) & 1) return HD_ERR_ARG;
    }
    // the median reads only the noisy input: source and destination must not overlap
    const uintptr_t s0 = (uintptr_t)img->src, s1 = s0 + (size_t)(img->H - 1) * img->src_pitch + row;
    const uintptr_t d0 = (uintptr_t)img->dst, d1 = d0 + (size_t)(img->H - 1) * img->dst_pitch + row;
    if (s0 < d1 && d0 < s1) return HD_ERR_ARG;
    if (need_amf) {
        const int s = img->p.smax;
        if (s < 3 || s > HD_SMAX_MAX || (s & 1) == 0) return HD_ERR_SMAX;
        if (img->p.unresolved != HD_UNRESOLVED_ZMED && img->p.unresolved != HD_UNRESOLVED_KEEP)
            return HD_ERR_ARG;
    }
    if (need_wiener) {
        const int w = img->p.wiener_w, wh = window_rows(img->p);
        if (w < 1 || w > HD_WIENER_W_MAX || (w & 1) == 0) return HD_ERR_WINDOW;
        if (wh < 1 || wh > HD_WIENER_W_MAX || (wh & 1) == 0) return HD_ERR_WINDOW;
        if (img->p.border != HD_BORDER_SYMMETRIC && img->p.border != HD_BORDER_ZERO) return HD_ERR_ARG;
        if (!(img->p.noise_var == img->p.noise_var)) return HD_ERR_ARG;   // NaN
        if (img->y_out && ((uintptr_t)img->y_out & 3)) return HD_ERR_ARG;
        if (img->noise_var_out && ((uintptr_t)img->noise_var_out & 7)) return HD_ERR_ARG;
    }
    (void)host_buffers;
    return HD_OK;
}

int device_sms()
{
    static std::mutex mu;
    static std::vector<int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lk(mu);
    if ((int)cache.size() <= dev) cache.resize(dev + 1, 0);
    if (cache[dev] == 0) cache[dev] = sm_count();
    return cache[dev];
}

size_t device_l2_bytes()
{
    static std::mutex mu;
    static std::vector<int> cache;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lk(mu);
    if ((int)cache.size() <= dev) cache.resize(dev + 1, -1);
    if (cache[dev] < 0) {
        int b = 0;
        if (cudaDeviceGetAttribute(&b, cudaDevAttrL2CacheSize, dev) != cudaSuccess) b = 0;
        cache[dev] = b;
    }
    return (size_t)cache[dev];
}

size_t f_pitch_of(int W, int dtype) { return round_up((size_t)W * elem_size(dtype), 16); }

// Workspace layout of a single image: [ticket][ImgCtl] [fbuf] [plane].  The
// plane (binary32 mu, s2 per pixel) is optional: without it phase 2
// recomputes the window sums from the f region.
size_t ctl_bytes() { return round_up(kTicketBytes + sizeof(ImgCtl), kAlign); }

size_t plane_bytes(int H, int W) { return round_up((size_t)H * (size_t)W * 2 * sizeof(float), kAlign); }

size_t single_ws_bytes(int H, int W, int dtype, bool needs_fbuf)
{
    size_t b = ctl_bytes();
    if (needs_fbuf) b += round_up((size_t)H * f_pitch_of(W, dtype), kAlign);
    return b;
}

size_t single_ws_full(int H, int W, int dtype, bool needs_fbuf)
{
    return single_ws_bytes(H, W, dtype, needs_fbuf) + plane_bytes(H, W);
}

ImgDesc make_desc(const hd_image *img, int mode, const hd_tuning &t, ImgCtl *ctl, uint8_t *fbuf,
                  float *plane = nullptr)
{
    ImgDesc d;
    std::memset(&d, 0, sizeof(d));
    d.src = static_cast<const uint8_t *>(img->src);
    d.dst = static_cast<uint8_t *>(img->dst);
    d.fbuf = fbuf;
    d.plane = plane;
    d.src_pitch = (long long)img->src_pitch;
    d.dst_pitch = (long long)img->dst_pitch;
    d.f_pitch = (long long)f_pitch_of(img->W, img->dtype);
    d.noise_var = img->p.noise_var;
    {
        // the host's IEEE division gives the correctly rounded reciprocal
        const double nw = (double)img->p.wiener_w * (double)window_rows(img->p);
        d.inv_den = 1.0 / (nw * nw * (double)img->H * (double)img->W);
    }
    d.noise_var_out = img->noise_var_out;
    d.y_out = img->y_out;
    d.ctl = ctl;
    d.H = img->H;
    d.W = img->W;
    d.elem = elem_size(img->dtype);
    d.maxv = (int)((1u << img->p.bits) - 1u);
    d.smax = img->p.smax;
    d.w = img->p.wiener_w;
    d.wh = window_rows(img->p);
    d.unresolved = img->p.unresolved;
    d.border_zero = img->p.border == HD_BORDER_ZERO;
    d.mode = mode;
    // same tile shape as the kernel: left margin rw rounded up to even, width even
    const int rw = mode == MODE_AMF ? 0 : img->p.wiener_w / 2;
    const int ry = mode == MODE_AMF ? 0 : window_rows(img->p) / 2;
    const int lm = rw + (rw & 1);
    const int TW = (64 - lm - rw) & ~1, TH = t.region_h - 2 * ry;
    d.tiles_x = (img->W + TW - 1) / TW;
    d.tiles_y = (img->H + TH - 1) / TH;
    d.p2_items = plane ? 0 : d.tiles_x * d.tiles_y;
    d.Hg = img->H;
    d.gy_off = 0;
    d.own0 = 0;
    d.own1 = img->H;
    return d;
}

// Same test as the kernel: 32-bit Wiener sums are exact when n * maxv < 2^17.
bool image_wide(const ImgDesc &d)
{
    if (d.mode == MODE_AMF) return false;
    const long long n = (long long)d.w * d.wh;
    return !(d.maxv < 0x8000 && (long long)(std::max(d.w, d.wh) + 1) * d.maxv <= 65535 && n * d.maxv < 131072);
}

int halo_a(const ImgDesc &d) { return (d.mode == MODE_AMF || d.mode == MODE_HYBRID_EST || d.mode == MODE_HYBRID_GIVEN) ? d.smax / 2 : 0; }

hd_status finish_params(LaunchParams &lp, const hd_tuning &t, int *grid, size_t *smem)
{
    lp.region_h = t.region_h;
    lp.small_growth = t.small_growth == 0 ? 32 : (t.small_growth < 0 ? 0 : t.small_growth);
    lp.select_lanes = t.select_lanes;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        lp.spin_limit = g_spin_limit;
    }
    *smem = smem_bytes(t.region_h, lp.ra_max, lp.wide);
    if (*smem > 227 * 1024) return HD_ERR_OVERFLOW;
    const int sms = device_sms();
    if (sms <= 0) return HD_ERR_CUDA;
    int per_sm = max_ctas_per_sm(*smem);
    if (per_sm <= 0) return HD_ERR_CUDA;
    if (t.ctas_per_sm > 0) per_sm = std::min(per_sm, t.ctas_per_sm);
    // plane mode: every resident CTA takes a share of the phase-2 pixels,
    // read straight from L2 when the plane, f and the output of the owned rows
    // fit in it (they were written moments before; measured faster up to a
    // 101 MB working set, slower from 154 MB), else staged by bulk copies,
    // which keep more bytes in flight from HBM
    if (lp.p2_plane) {
        const ImgDesc &d = lp.one;
        const size_t px = (size_t)(d.own1 - d.own0) * (size_t)d.W;
        lp.p2_direct = t.plane == 3 || (t.plane != 2 && px * (8 + 2 * (size_t)d.elem) <= device_l2_bytes());
    }
    *grid = std::max(1, lp.p2_plane ? sms * per_sm : std::min(lp.total_items, sms * per_sm));
    return HD_OK;
}

// Launch one image.  ws may be null for single-phase modes without a queue.
hd_status run_single(const hd_image *img, int mode, void *ws, size_t ws_bytes, cudaStream_t s)
{
    const hd_tuning t = current_tuning();
    const bool two_phase = mode == MODE_WIENER_EST || mode == MODE_HYBRID_EST;
    const bool needs_fbuf = mode == MODE_HYBRID_EST;
    ImgCtl *ctl = nullptr;
    unsigned int *ticket = nullptr;
    uint8_t *fbuf = nullptr;
    float *plane = nullptr;
    if (two_phase) {
        if (!ws || ((uintptr_t)ws % kAlign)) return HD_ERR_WORKSPACE;
        const size_t need = single_ws_bytes(img->H, img->W, img->dtype, needs_fbuf);
        if (ws_bytes < need) return HD_ERR_WORKSPACE;
        ticket = static_cast<unsigned int *>(ws);
        ctl = reinterpret_cast<ImgCtl *>(static_cast<uint8_t *>(ws) + kTicketBytes);
        if (needs_fbuf) fbuf = static_cast<uint8_t *>(ws) + ctl_bytes();
        if (t.plane != 1 && ws_bytes >= need + plane_bytes(img->H, img->W))
            plane = reinterpret_cast<float *>(static_cast<uint8_t *>(ws) + need);
    }
    LaunchParams lp;
    std::memset(&lp, 0, sizeof(lp));
    lp.descs = nullptr;
    lp.segs = nullptr;
    lp.one = make_desc(img, mode, t, ctl, fbuf, plane);
    const int tiles = lp.one.tiles_x * lp.one.tiles_y;
    lp.oneseg[0] = Seg{0, 1, 0, tiles};
    lp.nsegs = 1;
    lp.total_items = tiles;
    if (two_phase) {
        if (plane) {
            lp.p2_plane = 1;           // phase 2 runs after the queue, a share per CTA
        } else {
            lp.oneseg[1] = Seg{0, 2, tiles, lp.one.p2_items};
            lp.nsegs = 2;
            lp.total_items = tiles + lp.one.p2_items;
        }
        lp.ticket = ticket;
        lp.ctl_reset = ctl;
        lp.nctl = 1;
    }
    lp.ra_max = halo_a(lp.one);
    lp.wide = image_wide(lp.one);
    int grid = 0;
    size_t smem = 0;
    hd_status st = finish_params(lp, t, &grid, &smem);
    if (st != HD_OK) return st;
    if (launch_persistent(lp, grid, smem, (void *)s) != 0) return HD_ERR_CUDA;
    return HD_OK;
}

int hybrid_mode(const hd_image *img) { return img->p.noise_var < 0.0 ? MODE_HYBRID_EST : MODE_HYBRID_GIVEN; }

// ---------------------------------------------------------------- batches
struct BatchLayout {
    size_t ctl_off, desc_off, seg_off, fbuf_off, total;
    std::vector<size_t> fbuf_offsets;    // per image, or SIZE_MAX when not needed
    std::vector<size_t> plane_offsets;   // per image, or SIZE_MAX when not needed
};

BatchLayout batch_layout(const hd_image *imgs, int n)
{
    BatchLayout L;
    size_t off = kTicketBytes;
    L.ctl_off = off;
    off = round_up(off + sizeof(ImgCtl) * (size_t)n, kAlign);
    L.desc_off = off;
    off = round_up(off + sizeof(ImgDesc) * (size_t)n, kAlign);
    L.seg_off = off;
    off = round_up(off + sizeof(Seg) * (size_t)(2 * n), kAlign);
    L.fbuf_off = off;
    L.fbuf_offsets.resize(n);
    L.plane_offsets.resize(n);
    // a batch uses the recompute Wiener pass: an image's phase 2 already runs
    // beside the next image's phase 1, and a statistics plane per image would
    // add its traffic and slot overhead for no gain
    for (int i = 0; i < n; ++i) {
        L.plane_offsets[i] = SIZE_MAX;
        if (hybrid_mode(&imgs[i]) == MODE_HYBRID_EST) {
            L.fbuf_offsets[i] = off;
            off += round_up((size_t)imgs[i].H * f_pitch_of(imgs[i].W, imgs[i].dtype), kAlign);
        } else {
            L.fbuf_offsets[i] = SIZE_MAX;
        }
    }
    L.total = off;
    return L;
}

struct BatchTables {
    std::vector<ImgDesc> descs;
    std::vector<Seg> segs;
    int total_items = 0;
    int ra_max = 0, wide = 0;
    size_t table_bytes = 0;   // bytes from ctl_off to the end of the segment table
};

// Wiener tiles of an image are queued this many grids of tickets after its
// last median tile (see build_batch).
constexpr int kBatchLagGrids = 6;

// Grid of a batched launch with the current tuning (as finish_params sizes it).
long long batch_grid(const BatchTables &bt)
{
    const hd_tuning t = current_tuning();
    const size_t smem = smem_bytes(t.region_h, bt.ra_max, bt.wide);
    const int sms = device_sms();
    int per_sm = smem <= 227 * 1024 ? max_ctas_per_sm(smem) : 0;
    if (t.ctas_per_sm > 0 && per_sm > 0) per_sm = std::min(per_sm, t.ctas_per_sm);
    // no device answer (sizes only): a grid of one GB300 at 3 CTAs per SM
    if (sms <= 0 || per_sm <= 0) return 152LL * 3;
    return (long long)sms * per_sm;
}

hd_status build_batch(const hd_image *imgs, int n, void *ws, size_t ws_bytes, BatchTables &bt,
                      BatchLayout &L)
{
    if (!imgs || n < 1) return HD_ERR_ARG;
    if (n > (1 << 20)) return HD_ERR_OVERFLOW;
    for (int i = 0; i < n; ++i) {
        hd_status st = check_image(&imgs[i], true, true, false);
        if (st != HD_OK) return st;
    }
    L = batch_layout(imgs, n);
    if (!ws || ((uintptr_t)ws % kAlign)) return HD_ERR_WORKSPACE;
    if (ws_bytes < L.total) return HD_ERR_WORKSPACE;
    const hd_tuning t = current_tuning();
    uint8_t *base = static_cast<uint8_t *>(ws);
    ImgCtl *ctl = reinterpret_cast<ImgCtl *>(base + L.ctl_off);
    bt.descs.resize(n);
    for (int i = 0; i < n; ++i) {
        uint8_t *fb = L.fbuf_offsets[i] == SIZE_MAX ? nullptr : base + L.fbuf_offsets[i];
        float *pl = L.plane_offsets[i] == SIZE_MAX ? nullptr : reinterpret_cast<float *>(base + L.plane_offsets[i]);
        bt.descs[i] = make_desc(&imgs[i], hybrid_mode(&imgs[i]), t, ctl + i, fb, pl);
        bt.ra_max = std::max(bt.ra_max, halo_a(bt.descs[i]));
        bt.wide |= image_wide(bt.descs[i]) ? 1 : 0;
    }

    // ticket order: every image's median tiles (P1) in image order; an image's
    // Wiener tiles (P2) follow once `lag` more median tiles have been queued
    // after its last one, or at the end.  A P2 tile waits for all of its
    // image's P1 tiles, and those were handed out `lag` tickets earlier:
    // with lag a few times the grid, they are done by the time it starts,
    // so the wait is rarely more than one poll.
    const hd_tuning tn = current_tuning();
    const long long lag = (long long)(tn.batch_lag ? tn.batch_lag : kBatchLagGrids) * batch_grid(bt);
    long long first = 0;
    auto push = [&](int img, int phase) {
        const ImgDesc &d = bt.descs[img];
        const int items = phase == 1 ? d.tiles_x * d.tiles_y : d.p2_items;
        bt.segs.push_back(Seg{img, phase, (int)first, items});
        first += items;
    };
    // optionally the largest images first (the last images' Wiener tiles,
    // which cannot lag behind enough median tiles, then wait only for small
    // images' tails; measured no faster on the uneven 256-slice batch)
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    if (tn.batch_order == 1)
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            return (long long)bt.descs[a].H * bt.descs[a].W > (long long)bt.descs[b].H * bt.descs[b].W;
        });
    std::vector<long long> p1_end(n, 0);
    std::vector<int> pending;           // images whose P2 is not placed yet, in order
    size_t head = 0;
    for (int k = 0; k < n; ++k) {
        const int i = order[k];
        push(i, 1);
        p1_end[i] = first;
        if (mode_two_phase(bt.descs[i].mode)) pending.push_back(i);
        while (head < pending.size() && first - p1_end[pending[head]] >= lag) push(pending[head++], 2);
    }
    while (head < pending.size()) push(pending[head++], 2);
    if (first > 0x7fffffffLL) return HD_ERR_OVERFLOW;
    bt.total_items = (int)first;
    bt.table_bytes = L.seg_off + sizeof(Seg) * bt.segs.size() - L.ctl_off;
    return HD_OK;
}

LaunchParams batch_params(void *ws, const BatchLayout &L, const BatchTables &bt)
{
    uint8_t *base = static_cast<uint8_t *>(ws);
    LaunchParams lp;
    std::memset(&lp, 0, sizeof(lp));
    lp.descs = reinterpret_cast<const ImgDesc *>(base + L.desc_off);
    lp.segs = reinterpret_cast<const Seg *>(base + L.seg_off);
    lp.nsegs = (int)bt.segs.size();
    lp.total_items = bt.total_items;
    lp.ticket = reinterpret_cast<unsigned int *>(base);
    lp.ctl_reset = reinterpret_cast<ImgCtl *>(base + L.ctl_off);
    lp.nctl = (int)bt.descs.size();
    lp.ra_max = bt.ra_max;
    lp.wide = bt.wide;
    return lp;
}

// Host image of the descriptor + segment tables, laid out as in the workspace.
std::vector<uint8_t> table_image(const BatchLayout &L, const BatchTables &bt)
{
    std::vector<uint8_t> h(L.seg_off + sizeof(Seg) * bt.segs.size() - L.desc_off, 0);
    std::memcpy(h.data(), bt.descs.data(), sizeof(ImgDesc) * bt.descs.size());
    std::memcpy(h.data() + (L.seg_off - L.desc_off), bt.segs.data(), sizeof(Seg) * bt.segs.size());
    return h;
}

// ---------------------------------------------------------------- strips
// The listing's partitioned median (Algorithm 1, step 6 with `parts`
// sub-images): row strips [floor(i H / parts), floor((i+1) H / parts)), each
// median-filtered as an image of its own (borders reflect at the strip's
// edges), then the Wiener filter over the whole reassembled median image.
// Workspace: [median queue counters][Wiener workspace: its counters and control
// block, then the statistics plane when estimating][strip descriptors][strip
// segments][median image].  The offsets move with the image size and `parts`,
// so every call clears the control words it uses (one memset) before its
// launches: a workspace can serve calls of any size and partition in turn.
struct StripLayout {
    size_t wiener_off, desc_off, seg_off, fbuf_off, total;
    size_t control_bytes;     // [0, control_bytes) holds every counter of the call
};

StripLayout strip_layout(int H, int W, int dtype, const hd_params *p, int parts)
{
    StripLayout L;
    L.wiener_off = round_up(kTicketBytes, kAlign);
    L.control_bytes = L.wiener_off + ctl_bytes();
    const size_t wiener_bytes = p->noise_var < 0.0 ? single_ws_full(H, W, dtype, false) : ctl_bytes();
    L.desc_off = round_up(L.wiener_off + wiener_bytes, kAlign);
    L.seg_off = round_up(L.desc_off + sizeof(ImgDesc) * (size_t)parts, kAlign);
    L.fbuf_off = round_up(L.seg_off + sizeof(Seg) * (size_t)parts, kAlign);
    L.total = L.fbuf_off + round_up((size_t)H * f_pitch_of(W, dtype), kAlign);
    return L;
}

}  // namespace

namespace hd {
int hybrid_on_workspace(const void *img_, void *ws, size_t ws_bytes, void *stream)
{
    const hd_image *img = static_cast<const hd_image *>(img_);
    hd_status st = check_image(img, true, true, false);
    if (st != HD_OK) return st;
    return run_single(img, hybrid_mode(img), ws, ws_bytes, (cudaStream_t)stream);
}

int check_hybrid_image(const void *img) { return check_image(static_cast<const hd_image *>(img), true, true, false); }

size_t hybrid_control_bytes() { return ctl_bytes(); }

size_t hybrid_min_bytes(const void *img_)
{
    const hd_image *img = static_cast<const hd_image *>(img_);
    return img->p.noise_var < 0.0 ? single_ws_bytes(img->H, img->W, img->dtype, true) : 0;
}
}  // namespace hd

// A host pipeline keeps `depth` slots of device images (noisy in, result out)
// in the caller's workspace and three streams: host-to-device copies, kernels,
// device-to-host copies.  Step i uses slot i mod depth; events order the
// reuse of a slot after its previous step, so the copies of one step overlap
// the kernels of its neighbours.
struct hd_host_pipeline {
    int H = 0, W = 0, dtype = 0;
    hd_params p{};
    int depth = 0;
    uint8_t *ws = nullptr;
    size_t core = 0;          // bytes of the hybrid workspace at the start
    size_t plane = 0;         // bytes of one device image
    cudaStream_t h2d = nullptr, comp = nullptr, d2h = nullptr;
    std::vector<cudaEvent_t> ev_in, ev_k, ev_out;
    long long submitted = 0;
};

struct hd_batch_plan {
    void *ws = nullptr;
    LaunchParams lp;
    int grid = 0;
    size_t smem = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" {

hd_status amf_filter(const hd_image *img, hd_stream_t stream)
{
    hd_status st = check_image(img, true, false, false);
    if (st != HD_OK) return st;
    return run_single(img, MODE_AMF, nullptr, 0, (cudaStream_t)stream);
}

hd_status wiener_workspace_size(int H, int W, int dtype, const hd_params *p, size_t *bytes)
{
    if (!bytes || !p || H < 1 || W < 1) return HD_ERR_ARG;
    if (dtype != HD_U8 && dtype != HD_U16) return HD_ERR_DTYPE;
    *bytes = p->noise_var < 0.0 ? single_ws_full(H, W, dtype, false) : 0;
    return HD_OK;
}

hd_status wiener_filter(const hd_image *img, void *workspace, size_t ws_bytes, hd_stream_t stream)
{
    hd_status st = check_image(img, false, true, false);
    if (st != HD_OK) return st;
    const int mode = img->p.noise_var < 0.0 ? MODE_WIENER_EST : MODE_WIENER_GIVEN;
    return run_single(img, mode, workspace, ws_bytes, (cudaStream_t)stream);
}

hd_status hybrid_workspace_size(int H, int W, int dtype, const hd_params *p, size_t *bytes)
{
    if (!bytes || !p || H < 1 || W < 1) return HD_ERR_ARG;
    if (dtype != HD_U8 && dtype != HD_U16) return HD_ERR_DTYPE;
    *bytes = p->noise_var < 0.0 ? single_ws_full(H, W, dtype, true) : 0;
    return HD_OK;
}

hd_status hybrid_min_workspace_size(int H, int W, int dtype, const hd_params *p, size_t *bytes)
{
    if (!bytes || !p || H < 1 || W < 1) return HD_ERR_ARG;
    if (dtype != HD_U8 && dtype != HD_U16) return HD_ERR_DTYPE;
    *bytes = p->noise_var < 0.0 ? single_ws_bytes(H, W, dtype, true) : 0;
    return HD_OK;
}

hd_status hybrid_denoise(const hd_image *img, void *workspace, size_t ws_bytes, hd_stream_t stream)
{
    hd_status st = check_image(img, true, true, false);
    if (st != HD_OK) return st;
    return run_single(img, hybrid_mode(img), workspace, ws_bytes, (cudaStream_t)stream);
}

hd_status hybrid_host_workspace_size(int H, int W, int dtype, const hd_params *p, size_t *bytes)
{
    size_t b = 0;
    hd_status st = hybrid_workspace_size(H, W, dtype, p, &b);
    if (st != HD_OK) return st;
    const size_t plane = round_up((size_t)H * (size_t)W * elem_size(dtype), kAlign);
    *bytes = round_up(b, kAlign) + 2 * plane;
    return HD_OK;
}

hd_status hybrid_denoise_host(const hd_image *img, void *workspace, size_t ws_bytes, hd_stream_t stream)
{
    hd_status st = check_image(img, true, true, true);
    if (st != HD_OK) return st;
    size_t need = 0;
    hybrid_host_workspace_size(img->H, img->W, img->dtype, &img->p, &need);
    if (!workspace || ((uintptr_t)workspace % kAlign)) return HD_ERR_WORKSPACE;
    if (ws_bytes < need) return HD_ERR_WORKSPACE;
    size_t core = 0;
    hybrid_workspace_size(img->H, img->W, img->dtype, &img->p, &core);
    core = round_up(core, kAlign);
    // device planes at the tight row pitch: a tight host buffer then moves as
    // one linear copy each way (a pitched copy moves row by row)
    const size_t row = (size_t)img->W * elem_size(img->dtype);
    const size_t pitch = row;
    const size_t plane = round_up((size_t)img->H * pitch, kAlign);
    uint8_t *base = static_cast<uint8_t *>(workspace);
    uint8_t *dsrc = base + core;
    uint8_t *ddst = dsrc + plane;
    cudaStream_t s = (cudaStream_t)stream;
    const cudaError_t ein = img->src_pitch == row
                                ? cudaMemcpyAsync(dsrc, img->src, row * img->H, cudaMemcpyHostToDevice, s)
                                : cudaMemcpy2DAsync(dsrc, pitch, img->src, img->src_pitch, row, img->H,
                                                    cudaMemcpyHostToDevice, s);
    if (ein != cudaSuccess) return HD_ERR_CUDA;
    hd_image dimg = *img;
    dimg.src = dsrc;
    dimg.dst = ddst;
    dimg.src_pitch = pitch;
    dimg.dst_pitch = pitch;
    st = run_single(&dimg, hybrid_mode(&dimg), core ? workspace : nullptr, core, s);
    if (st != HD_OK) return st;
    const cudaError_t eout = img->dst_pitch == row
                                 ? cudaMemcpyAsync(img->dst, ddst, row * img->H, cudaMemcpyDeviceToHost, s)
                                 : cudaMemcpy2DAsync(img->dst, img->dst_pitch, ddst, pitch, row, img->H,
                                                     cudaMemcpyDeviceToHost, s);
    if (eout != cudaSuccess) return HD_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return HD_ERR_CUDA;
    return HD_OK;
}

hd_status hybrid_strips_workspace_size(int H, int W, int dtype, const hd_params *p, int parts, size_t *bytes)
{
    if (!bytes || !p || H < 1 || W < 1) return HD_ERR_ARG;
    if (dtype != HD_U8 && dtype != HD_U16) return HD_ERR_DTYPE;
    if (parts < 1 || parts > H) return HD_ERR_ARG;
    if (parts == 1) return hybrid_workspace_size(H, W, dtype, p, bytes);
    *bytes = strip_layout(H, W, dtype, p, parts).total;
    return HD_OK;
}

hd_status hybrid_denoise_strips(const hd_image *img, int parts, void *workspace, size_t ws_bytes,
                                hd_stream_t stream)
{
    hd_status st = check_image(img, true, true, false);
    if (st != HD_OK) return st;
    if (parts < 1 || parts > img->H) return HD_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (parts == 1) {
        // the whole-image hybrid, on the same workspace: clear its counters first
        if (workspace && ((uintptr_t)workspace % kAlign) == 0 && ws_bytes >= ctl_bytes() &&
            cudaMemsetAsync(workspace, 0, ctl_bytes(), s) != cudaSuccess)
            return HD_ERR_CUDA;
        return run_single(img, hybrid_mode(img), workspace, ws_bytes, s);
    }
    const StripLayout L = strip_layout(img->H, img->W, img->dtype, &img->p, parts);
    if (!workspace || ((uintptr_t)workspace % kAlign)) return HD_ERR_WORKSPACE;
    if (ws_bytes < L.total) return HD_ERR_WORKSPACE;
    uint8_t *base = static_cast<uint8_t *>(workspace);
    uint8_t *fbuf = base + L.fbuf_off;
    const size_t f_pitch = f_pitch_of(img->W, img->dtype);
    const hd_tuning t = current_tuning();

    // the medians of all strips in one persistent launch
    std::vector<uint8_t> tab(L.seg_off - L.desc_off + sizeof(Seg) * (size_t)parts, 0);
    ImgDesc *descs = reinterpret_cast<ImgDesc *>(tab.data());
    Seg *segs = reinterpret_cast<Seg *>(tab.data() + (L.seg_off - L.desc_off));
    long long first = 0;
    for (int i = 0; i < parts; ++i) {
        const int y0 = (int)((long long)i * img->H / parts), y1 = (int)((long long)(i + 1) * img->H / parts);
        hd_image si = *img;
        si.src = static_cast<const uint8_t *>(img->src) + (size_t)y0 * img->src_pitch;
        si.dst = fbuf + (size_t)y0 * f_pitch;
        si.dst_pitch = f_pitch;
        si.H = y1 - y0;
        si.noise_var_out = nullptr;
        si.y_out = nullptr;
        descs[i] = make_desc(&si, MODE_AMF, t, nullptr, nullptr);
        const int tiles = descs[i].tiles_x * descs[i].tiles_y;
        segs[i] = Seg{i, 1, (int)first, tiles};
        first += tiles;
    }
    if (first > 0x7fffffffLL) return HD_ERR_OVERFLOW;
    LaunchParams lp;
    std::memset(&lp, 0, sizeof(lp));
    lp.descs = reinterpret_cast<const ImgDesc *>(base + L.desc_off);
    lp.segs = reinterpret_cast<const Seg *>(base + L.seg_off);
    lp.nsegs = parts;
    lp.total_items = (int)first;
    lp.ticket = reinterpret_cast<unsigned int *>(base);
    lp.ra_max = img->p.smax / 2;
    int grid = 0;
    size_t smem = 0;
    st = finish_params(lp, t, &grid, &smem);
    if (st != HD_OK) return st;
    if (cudaMemsetAsync(base, 0, L.control_bytes, s) != cudaSuccess) return HD_ERR_CUDA;
    if (launch_table_upload(base + L.desc_off, tab.data(), tab.size(), (void *)s) != 0) return HD_ERR_CUDA;
    if (launch_persistent(lp, grid, smem, (void *)s) != 0) return HD_ERR_CUDA;

    // the Wiener filter of the whole median image
    hd_image fi = *img;
    fi.src = fbuf;
    fi.src_pitch = f_pitch;
    const int mode = img->p.noise_var < 0.0 ? MODE_WIENER_EST : MODE_WIENER_GIVEN;
    return run_single(&fi, mode, base + L.wiener_off, L.desc_off - L.wiener_off, s);
}

static size_t pipeline_plane(int H, int W, int dtype)
{
    return round_up((size_t)H * (size_t)W * elem_size(dtype), kAlign);
}

hd_status hd_host_pipeline_workspace_size(int H, int W, int dtype, const hd_params *p, int depth, size_t *bytes)
{
    if (!bytes || depth < 1 || depth > HD_PIPELINE_DEPTH_MAX) return HD_ERR_ARG;
    size_t b = 0;
    hd_status st = hybrid_workspace_size(H, W, dtype, p, &b);
    if (st != HD_OK) return st;
    *bytes = round_up(b, kAlign) + 2 * (size_t)depth * pipeline_plane(H, W, dtype);
    return HD_OK;
}

static void pipeline_release(hd_host_pipeline *pl)
{
    if (pl->comp) cudaStreamSynchronize(pl->comp);
    if (pl->h2d) cudaStreamSynchronize(pl->h2d);
    if (pl->d2h) cudaStreamSynchronize(pl->d2h);
    for (auto *v : {&pl->ev_in, &pl->ev_k, &pl->ev_out})
        for (cudaEvent_t e : *v)
            if (e) cudaEventDestroy(e);
    for (cudaStream_t st : {pl->h2d, pl->comp, pl->d2h})
        if (st) cudaStreamDestroy(st);
    delete pl;
}

hd_status hd_host_pipeline_create(int H, int W, int dtype, const hd_params *p, int depth, void *workspace,
                                  size_t ws_bytes, hd_host_pipeline **out)
{
    if (!out || !p) return HD_ERR_ARG;
    *out = nullptr;
    size_t need = 0;
    hd_status st = hd_host_pipeline_workspace_size(H, W, dtype, p, depth, &need);
    if (st != HD_OK) return st;
    if (!workspace || ((uintptr_t)workspace % kAlign) || ws_bytes < need) return HD_ERR_WORKSPACE;
    hd_host_pipeline *pl = new (std::nothrow) hd_host_pipeline();
    if (!pl) return HD_ERR_ARG;
    pl->H = H;
    pl->W = W;
    pl->dtype = dtype;
    pl->p = *p;
    pl->depth = depth;
    pl->ws = static_cast<uint8_t *>(workspace);
    size_t core = 0;
    hybrid_workspace_size(H, W, dtype, p, &core);
    pl->core = round_up(core, kAlign);
    pl->plane = pipeline_plane(H, W, dtype);
    // the parameters are checked once, on slot 0's images
    hd_image img;
    std::memset(&img, 0, sizeof(img));
    img.src = pl->ws + pl->core;
    img.dst = pl->ws + pl->core + pl->plane;
    img.H = H;
    img.W = W;
    img.src_pitch = img.dst_pitch = (size_t)W * elem_size(dtype);
    img.dtype = dtype;
    img.p = *p;
    st = check_image(&img, true, true, false);
    if (st != HD_OK) {
        delete pl;
        return st;
    }
    bool ok = true;
    for (cudaStream_t *sp : {&pl->h2d, &pl->comp, &pl->d2h})
        ok = ok && cudaStreamCreateWithFlags(sp, cudaStreamNonBlocking) == cudaSuccess;
    for (auto *v : {&pl->ev_in, &pl->ev_k, &pl->ev_out}) {
        v->assign(depth, nullptr);
        for (cudaEvent_t &e : *v) ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
        pipeline_release(pl);
        cudaGetLastError();
        return HD_ERR_CUDA;
    }
    *out = pl;
    return HD_OK;
}

hd_status hd_host_pipeline_submit(hd_host_pipeline *pl, const void *src, size_t src_pitch, void *dst,
                                  size_t dst_pitch)
{
    if (!pl || !src || !dst) return HD_ERR_ARG;
    const size_t row = (size_t)pl->W * elem_size(pl->dtype);
    if (src_pitch < row || dst_pitch < row) return HD_ERR_ARG;
    const int s = (int)(pl->submitted % pl->depth);
    uint8_t *dsrc = pl->ws + pl->core + 2 * (size_t)s * pl->plane;
    uint8_t *ddst = dsrc + pl->plane;
    const size_t H = (size_t)pl->H;
    // in: after the slot's previous kernel has read its noisy image
    if (cudaStreamWaitEvent(pl->h2d, pl->ev_k[s], 0) != cudaSuccess) return HD_ERR_CUDA;
    const cudaError_t ein = src_pitch == row
                                ? cudaMemcpyAsync(dsrc, src, row * H, cudaMemcpyHostToDevice, pl->h2d)
                                : cudaMemcpy2DAsync(dsrc, row, src, src_pitch, row, H, cudaMemcpyHostToDevice,
                                                    pl->h2d);
    if (ein != cudaSuccess || cudaEventRecord(pl->ev_in[s], pl->h2d) != cudaSuccess) return HD_ERR_CUDA;
    // kernel: after the copy in, and after the slot's previous result has left
    if (cudaStreamWaitEvent(pl->comp, pl->ev_in[s], 0) != cudaSuccess) return HD_ERR_CUDA;
    if (cudaStreamWaitEvent(pl->comp, pl->ev_out[s], 0) != cudaSuccess) return HD_ERR_CUDA;
    hd_image img;
    std::memset(&img, 0, sizeof(img));
    img.src = dsrc;
    img.dst = ddst;
    img.H = pl->H;
    img.W = pl->W;
    img.src_pitch = img.dst_pitch = row;
    img.dtype = pl->dtype;
    img.p = pl->p;
    hd_status st = run_single(&img, hybrid_mode(&img), pl->core ? pl->ws : nullptr, pl->core, pl->comp);
    if (st != HD_OK) return st;
    if (cudaEventRecord(pl->ev_k[s], pl->comp) != cudaSuccess) return HD_ERR_CUDA;
    // out: after the kernel
    if (cudaStreamWaitEvent(pl->d2h, pl->ev_k[s], 0) != cudaSuccess) return HD_ERR_CUDA;
    const cudaError_t eout = dst_pitch == row
                                 ? cudaMemcpyAsync(dst, ddst, row * H, cudaMemcpyDeviceToHost, pl->d2h)
                                 : cudaMemcpy2DAsync(dst, dst_pitch, ddst, row, row, H, cudaMemcpyDeviceToHost,
                                                     pl->d2h);
    if (eout != cudaSuccess || cudaEventRecord(pl->ev_out[s], pl->d2h) != cudaSuccess) return HD_ERR_CUDA;
    ++pl->submitted;
    return HD_OK;
}

hd_status hd_host_pipeline_wait(hd_host_pipeline *pl)
{
    if (!pl) return HD_ERR_ARG;
    bool ok = cudaStreamSynchronize(pl->h2d) == cudaSuccess;
    ok = cudaStreamSynchronize(pl->comp) == cudaSuccess && ok;
    ok = cudaStreamSynchronize(pl->d2h) == cudaSuccess && ok;
    return ok ? HD_OK : HD_ERR_CUDA;
}

hd_status hd_host_pipeline_destroy(hd_host_pipeline *pl)
{
    if (!pl) return HD_ERR_ARG;
    pipeline_release(pl);
    return HD_OK;
}

hd_status hybrid_batched_workspace_size(const hd_image *imgs, int n, size_t *bytes)
{
    if (!imgs || n < 1 || !bytes) return HD_ERR_ARG;
    *bytes = batch_layout(imgs, n).total;
    return HD_OK;
}

hd_status hybrid_denoise_batched(const hd_image *imgs, int n, void *workspace, size_t ws_bytes,
                                 hd_stream_t stream)
{
    BatchTables bt;
    BatchLayout L;
    hd_status st = build_batch(imgs, n, workspace, ws_bytes, bt, L);
    if (st != HD_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<uint8_t> h = table_image(L, bt);
    uint8_t *base = static_cast<uint8_t *>(workspace);
    LaunchParams lp = batch_params(workspace, L, bt);
    int grid = 0;
    size_t smem = 0;
    st = finish_params(lp, current_tuning(), &grid, &smem);
    if (st != HD_OK) return st;
    // the tables travel in kernel parameters: nothing here waits for the stream
    if (launch_table_upload(base + L.desc_off, h.data(), h.size(), (void *)s) != 0) return HD_ERR_CUDA;
    if (cudaMemsetAsync(base, 0, L.desc_off, s) != cudaSuccess) return HD_ERR_CUDA;
    if (launch_persistent(lp, grid, smem, (void *)s) != 0) return HD_ERR_CUDA;
    return HD_OK;
}

hd_status hd_batch_plan_create(const hd_image *imgs, int n, void *workspace, size_t ws_bytes,
                               hd_batch_plan **plan)
{
    if (!plan) return HD_ERR_ARG;
    *plan = nullptr;
    BatchTables bt;
    BatchLayout L;
    hd_status st = build_batch(imgs, n, workspace, ws_bytes, bt, L);
    if (st != HD_OK) return st;
    std::vector<uint8_t> h = table_image(L, bt);
    uint8_t *base = static_cast<uint8_t *>(workspace);
    if (cudaMemcpy(base + L.desc_off, h.data(), h.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return HD_ERR_CUDA;
    if (cudaMemset(base, 0, L.desc_off) != cudaSuccess) return HD_ERR_CUDA;
    hd_batch_plan *p = new (std::nothrow) hd_batch_plan();
    if (!p) return HD_ERR_ARG;
    p->ws = workspace;
    p->lp = batch_params(workspace, L, bt);
    st = finish_params(p->lp, current_tuning(), &p->grid, &p->smem);
    if (st != HD_OK) {
        delete p;
        return st;
    }
    // record the kernel as a graph on a private capture stream
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        delete p;
        return HD_ERR_CUDA;
    }
    bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) ok = launch_persistent(p->lp, p->grid, p->smem, (void *)cs) == 0;
    cudaGraph_t g = nullptr;
    const bool ended = cudaStreamEndCapture(cs, &g) == cudaSuccess;
    ok = ok && ended && g;
    if (ok) ok = cudaGraphInstantiate(&p->exec, g, 0) == cudaSuccess;
    cudaStreamDestroy(cs);
    p->graph = g;
    if (!ok) {
        if (p->exec) cudaGraphExecDestroy(p->exec);
        if (p->graph) cudaGraphDestroy(p->graph);
        delete p;
        cudaGetLastError();
        return HD_ERR_CUDA;
    }
    *plan = p;
    return HD_OK;
}

hd_status hd_batch_plan_launch(hd_batch_plan *plan, hd_stream_t stream)
{
    if (!plan || !plan->exec) return HD_ERR_ARG;
    if (cudaGraphLaunch(plan->exec, (cudaStream_t)stream) != cudaSuccess) return HD_ERR_CUDA;
    return HD_OK;
}

hd_status hd_batch_plan_destroy(hd_batch_plan *plan)
{
    if (!plan) return HD_ERR_ARG;
    if (plan->exec) cudaGraphExecDestroy(plan->exec);
    if (plan->graph) cudaGraphDestroy(plan->graph);
    delete plan;
    return HD_OK;
}

// A batch pipeline keeps `depth` slots, each with device planes for every
// image of the batch (noisy in, result out) and its own batch plan over them,
// and three streams as the host pipeline does: step i uses slot i mod depth,
// and events order a slot's reuse after its previous step.
struct BatchPipeLayout {
    std::vector<size_t> off;      // per image: offset of its plane within a slot's plane area
    std::vector<size_t> bytes;    // per image: H * W * element size (tight rows)
    size_t planes = 0;            // bytes of one plane area (all images)
    size_t batch_ws = 0;          // bytes of one slot's batch workspace
    size_t slot = 0;              // bytes of one slot: [batch workspace][noisy planes][result planes]
};

static hd_status batch_pipe_layout(const hd_image *imgs, int n, BatchPipeLayout &L)
{
    if (!imgs || n < 1) return HD_ERR_ARG;
    if (n > (1 << 20)) return HD_ERR_OVERFLOW;
    L.off.resize(n);
    L.bytes.resize(n);
    size_t o = 0;
    for (int i = 0; i < n; ++i) {
        const hd_image &im = imgs[i];
        if (im.dtype != HD_U8 && im.dtype != HD_U16) return HD_ERR_DTYPE;
        if (im.H < 1 || im.W < 1) return HD_ERR_ARG;
        if (im.H > HD_DIM_MAX || im.W > HD_DIM_MAX) return HD_ERR_OVERFLOW;
        const size_t es = (size_t)elem_size(im.dtype);
        // planes packed back to back, each aligned to its element size: a batch
        // of one dtype is one contiguous run (one copy when the host side is too)
        o = round_up(o, es);
        L.off[i] = o;
        L.bytes[i] = (size_t)im.H * (size_t)im.W * es;
        o += L.bytes[i];
    }
    L.planes = round_up(o, kAlign);
    L.batch_ws = round_up(batch_layout(imgs, n).total, kAlign);
    L.slot = L.batch_ws + 2 * L.planes;
    return HD_OK;
}

struct hd_batch_pipeline {
    int n = 0, depth = 0;
    BatchPipeLayout L;
    std::vector<size_t> row;      // per image: W * element size
    std::vector<int> H;
    uint8_t *ws = nullptr;
    std::vector<hd_batch_plan *> plans;
    cudaStream_t h2d = nullptr, comp = nullptr, d2h = nullptr;
    std::vector<cudaEvent_t> ev_in, ev_k, ev_out;
    long long submitted = 0;
};

static void batch_pipe_release(hd_batch_pipeline *pl)
{
    for (cudaStream_t st : {pl->comp, pl->h2d, pl->d2h})
        if (st) cudaStreamSynchronize(st);
    for (hd_batch_plan *p : pl->plans)
        if (p) hd_batch_plan_destroy(p);
    for (auto *v : {&pl->ev_in, &pl->ev_k, &pl->ev_out})
        for (cudaEvent_t e : *v)
            if (e) cudaEventDestroy(e);
    for (cudaStream_t st : {pl->h2d, pl->comp, pl->d2h})
        if (st) cudaStreamDestroy(st);
    delete pl;
}

// Copies of one direction for all images of a slot: runs of images whose host
// rows are tight and whose host and device planes both follow each other
// without a gap move as one copy; any other image moves on its own.
static hd_status batch_pipe_copies(const hd_batch_pipeline *pl, uint8_t *dev_area, const void *const *host,
                                   const size_t *pitch, bool to_device, cudaStream_t s)
{
    const int n = pl->n;
    const uint8_t *run_host = nullptr;
    uint8_t *run_dev = nullptr;
    size_t run_len = 0;
    auto flush = [&]() -> bool {
        if (!run_len) return true;
        const cudaError_t e =
            to_device ? cudaMemcpyAsync(run_dev, run_host, run_len, cudaMemcpyHostToDevice, s)
                      : cudaMemcpyAsync(const_cast<uint8_t *>(run_host), run_dev, run_len, cudaMemcpyDeviceToHost, s);
        run_len = 0;
        return e == cudaSuccess;
    };
    for (int i = 0; i < n; ++i) {
        const uint8_t *h = static_cast<const uint8_t *>(host[i]);
        uint8_t *d = dev_area + pl->L.off[i];
        const size_t row = pl->row[i], bytes = pl->L.bytes[i];
        if (pitch[i] == row) {
            if (run_len && h == run_host + run_len && d == run_dev + run_len) {
                run_len += bytes;
                continue;
            }
            if (!flush()) return HD_ERR_CUDA;
            run_host = h;
            run_dev = d;
            run_len = bytes;
            continue;
        }
        if (!flush()) return HD_ERR_CUDA;
        const cudaError_t e =
            to_device ? cudaMemcpy2DAsync(d, row, h, pitch[i], row, (size_t)pl->H[i], cudaMemcpyHostToDevice, s)
                      : cudaMemcpy2DAsync(const_cast<uint8_t *>(h), pitch[i], d, row, row, (size_t)pl->H[i],
                                          cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return HD_ERR_CUDA;
    }
    return flush() ? HD_OK : HD_ERR_CUDA;
}

hd_status hd_batch_pipeline_workspace_size(const hd_image *imgs, int n, int depth, size_t *bytes)
{
    if (!bytes || depth < 1 || depth > HD_PIPELINE_DEPTH_MAX) return HD_ERR_ARG;
    BatchPipeLayout L;
    hd_status st = batch_pipe_layout(imgs, n, L);
    if (st != HD_OK) return st;
    *bytes = (size_t)depth * L.slot;
    return HD_OK;
}

hd_status hd_batch_pipeline_create(const hd_image *imgs, int n, int depth, void *workspace, size_t ws_bytes,
                                   hd_batch_pipeline **out)
{
    if (!out) return HD_ERR_ARG;
    *out = nullptr;
    size_t need = 0;
    hd_status st = hd_batch_pipeline_workspace_size(imgs, n, depth, &need);
    if (st != HD_OK) return st;
    if (!workspace || ((uintptr_t)workspace % kAlign) || ws_bytes < need) return HD_ERR_WORKSPACE;
    hd_batch_pipeline *pl = new (std::nothrow) hd_batch_pipeline();
    if (!pl) return HD_ERR_ARG;
    pl->n = n;
    pl->depth = depth;
    batch_pipe_layout(imgs, n, pl->L);
    pl->ws = static_cast<uint8_t *>(workspace);
    pl->row.resize(n);
    pl->H.resize(n);
    for (int i = 0; i < n; ++i) {
        pl->row[i] = (size_t)imgs[i].W * elem_size(imgs[i].dtype);
        pl->H[i] = imgs[i].H;
    }
    // one batch plan per slot over that slot's device planes (the plan checks
    // every image's parameters)
    std::vector<hd_image> dimgs(imgs, imgs + n);
    pl->plans.assign(depth, nullptr);
    for (int k = 0; k < depth && st == HD_OK; ++k) {
        uint8_t *slot = pl->ws + (size_t)k * pl->L.slot;
        uint8_t *in = slot + pl->L.batch_ws, *res = in + pl->L.planes;
        for (int i = 0; i < n; ++i) {
            dimgs[i].src = in + pl->L.off[i];
            dimgs[i].dst = res + pl->L.off[i];
            dimgs[i].src_pitch = dimgs[i].dst_pitch = pl->row[i];
            dimgs[i].noise_var_out = nullptr;
            dimgs[i].y_out = nullptr;
        }
        st = hd_batch_plan_create(dimgs.data(), n, slot, pl->L.batch_ws, &pl->plans[k]);
    }
    if (st != HD_OK) {
        batch_pipe_release(pl);
        return st;
    }
    bool ok = true;
    for (cudaStream_t *sp : {&pl->h2d, &pl->comp, &pl->d2h})
        ok = ok && cudaStreamCreateWithFlags(sp, cudaStreamNonBlocking) == cudaSuccess;
    for (auto *v : {&pl->ev_in, &pl->ev_k, &pl->ev_out}) {
        v->assign(depth, nullptr);
        for (cudaEvent_t &e : *v) ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
        batch_pipe_release(pl);
        cudaGetLastError();
        return HD_ERR_CUDA;
    }
    *out = pl;
    return HD_OK;
}

hd_status hd_batch_pipeline_submit(hd_batch_pipeline *pl, const void *const *srcs, const size_t *src_pitches,
                                   void *const *dsts, const size_t *dst_pitches)
{
    if (!pl || !srcs || !src_pitches || !dsts || !dst_pitches) return HD_ERR_ARG;
    for (int i = 0; i < pl->n; ++i) {
        if (!srcs[i] || !dsts[i]) return HD_ERR_ARG;
        if (src_pitches[i] < pl->row[i] || dst_pitches[i] < pl->row[i]) return HD_ERR_ARG;
    }
    const int k = (int)(pl->submitted % pl->depth);
    uint8_t *slot = pl->ws + (size_t)k * pl->L.slot;
    uint8_t *in = slot + pl->L.batch_ws, *res = in + pl->L.planes;
    // in: after the slot's previous kernel has read its noisy planes
    if (cudaStreamWaitEvent(pl->h2d, pl->ev_k[k], 0) != cudaSuccess) return HD_ERR_CUDA;
    hd_status st = batch_pipe_copies(pl, in, srcs, src_pitches, true, pl->h2d);
    if (st != HD_OK) return st;
    if (cudaEventRecord(pl->ev_in[k], pl->h2d) != cudaSuccess) return HD_ERR_CUDA;
    // kernel: after the copies in, and after the slot's previous results have left
    if (cudaStreamWaitEvent(pl->comp, pl->ev_in[k], 0) != cudaSuccess) return HD_ERR_CUDA;
    if (cudaStreamWaitEvent(pl->comp, pl->ev_out[k], 0) != cudaSuccess) return HD_ERR_CUDA;
    st = hd_batch_plan_launch(pl->plans[k], pl->comp);
    if (st != HD_OK) return st;
    if (cudaEventRecord(pl->ev_k[k], pl->comp) != cudaSuccess) return HD_ERR_CUDA;
    // out: after the kernel
    if (cudaStreamWaitEvent(pl->d2h, pl->ev_k[k], 0) != cudaSuccess) return HD_ERR_CUDA;
    st = batch_pipe_copies(pl, res, const_cast<const void *const *>(dsts), dst_pitches, false, pl->d2h);
    if (st != HD_OK) return st;
    if (cudaEventRecord(pl->ev_out[k], pl->d2h) != cudaSuccess) return HD_ERR_CUDA;
    ++pl->submitted;
    return HD_OK;
}

hd_status hd_batch_pipeline_wait(hd_batch_pipeline *pl)
{
    if (!pl) return HD_ERR_ARG;
    bool ok = cudaStreamSynchronize(pl->h2d) == cudaSuccess;
    ok = cudaStreamSynchronize(pl->comp) == cudaSuccess && ok;
    ok = cudaStreamSynchronize(pl->d2h) == cudaSuccess && ok;
    return ok ? HD_OK : HD_ERR_CUDA;
}

hd_status hd_batch_pipeline_destroy(hd_batch_pipeline *pl)
{
    if (!pl) return HD_ERR_ARG;
    batch_pipe_release(pl);
    return HD_OK;
}

// ---------------------------------------------------------------- image parts
// One image split by row strips, one part per GPU.  A part's workspace:
// [queue counters + control block][median plane of the buffer rows]
// [statistics plane of the buffer rows, 16 bytes to spare].
static size_t part_plane_bytes(const hd_part *pt)
{
    return round_up((size_t)pt->buf_rows * (size_t)pt->W * 2 * sizeof(float) + 16, kAlign);
}

static hd_status check_part(const hd_part *pt, bool need_dst)
{
    if (!pt) return HD_ERR_ARG;
    if (pt->dtype != HD_U8 && pt->dtype != HD_U16) return HD_ERR_DTYPE;
    if (pt->dtype == HD_U8 && pt->p.bits != 8) return HD_ERR_DTYPE;
    if (pt->dtype == HD_U16 && (pt->p.bits < 1 || pt->p.bits > 16)) return HD_ERR_DTYPE;
    if (pt->H < 1 || pt->W < 1) return HD_ERR_ARG;
    if (pt->H > HD_DIM_MAX || pt->W > HD_DIM_MAX) return HD_ERR_OVERFLOW;
    const int s = pt->p.smax, w = pt->p.wiener_w, wh = window_rows(pt->p);
    if (s < 3 || s > HD_SMAX_MAX || (s & 1) == 0) return HD_ERR_SMAX;
    if (w < 1 || w > HD_WIENER_W_MAX || (w & 1) == 0) return HD_ERR_WINDOW;
    if (wh < 1 || wh > HD_WIENER_W_MAX || (wh & 1) == 0) return HD_ERR_WINDOW;
    if (pt->p.unresolved != HD_UNRESOLVED_ZMED && pt->p.unresolved != HD_UNRESOLVED_KEEP) return HD_ERR_ARG;
    if (pt->p.border != HD_BORDER_SYMMETRIC && pt->p.border != HD_BORDER_ZERO) return HD_ERR_ARG;
    // only the estimated noise variance needs the exchange of sums
    if (!(pt->p.noise_var < 0.0)) return HD_ERR_ARG;
    // rows: the part's own rows inside its buffer, the buffer inside the image,
    // and the buffer holding every halo row the own rows' windows read
    const int h = s / 2 + wh / 2;
    if (pt->buf_row0 < 0 || pt->buf_rows < 1 || pt->buf_row0 + pt->buf_rows > pt->H) return HD_ERR_ARG;
    if (pt->own_rows < 1 || pt->own_row0 < pt->buf_row0 ||
        pt->own_row0 + pt->own_rows > pt->buf_row0 + pt->buf_rows)
        return HD_ERR_ARG;
    if (pt->buf_row0 > std::max(0, pt->own_row0 - h)) return HD_ERR_ARG;
    if (pt->buf_row0 + pt->buf_rows < std::min(pt->H, pt->own_row0 + pt->own_rows + h)) return HD_ERR_ARG;
    const size_t es = (size_t)elem_size(pt->dtype), row = (size_t)pt->W * es;
    if (!pt->src || pt->src_pitch < row) return HD_ERR_ARG;
    if (es == 2 && (((uintptr_t)pt->src | pt->src_pitch) & 1)) return HD_ERR_ARG;
    if (need_dst) {
        if (!pt->dst || pt->dst_pitch < row) return HD_ERR_ARG;
        if (es == 2 && (((uintptr_t)pt->dst | pt->dst_pitch) & 1)) return HD_ERR_ARG;
        const uintptr_t s0 = (uintptr_t)pt->src, s1 = s0 + (size_t)(pt->buf_rows - 1) * pt->src_pitch + row;
        const uintptr_t d0 = (uintptr_t)pt->dst, d1 = d0 + (size_t)(pt->own_rows - 1) * pt->dst_pitch + row;
        if (s0 < d1 && d0 < s1) return HD_ERR_ARG;
    }
    return HD_OK;
}

// The descriptor of a part: the buffer as the image, the own rows as the
// tiled and applied range, the whole image's rows for M(q) and the noise
// variance's denominator.
static ImgDesc part_desc(const hd_part *pt, const hd_tuning &t, uint8_t *ws)
{
    hd_image img;
    std::memset(&img, 0, sizeof(img));
    img.src = pt->src;
    img.dst = pt->dst;
    img.H = pt->buf_rows;
    img.W = pt->W;
    img.src_pitch = pt->src_pitch;
    img.dst_pitch = pt->dst_pitch;
    img.dtype = pt->dtype;
    img.p = pt->p;
    ImgCtl *ctl = reinterpret_cast<ImgCtl *>(ws + kTicketBytes);
    uint8_t *fbuf = ws + ctl_bytes();
    const size_t fb = round_up((size_t)pt->buf_rows * f_pitch_of(pt->W, pt->dtype), kAlign);
    const int own0 = pt->own_row0 - pt->buf_row0;
    // the plane base sits 8 bytes past a 16-byte boundary when the first owned
    // pixel's index is odd, so that pixel's (mu, s2) pair is 16-byte aligned
    const size_t shift = ((size_t)own0 * (size_t)pt->W) & 1 ? 8 : 0;
    float *plane = reinterpret_cast<float *>(ws + ctl_bytes() + fb + shift);
    ImgDesc d = make_desc(&img, MODE_HYBRID_EST, t, ctl, fbuf, plane);
    d.Hg = pt->H;
    d.gy_off = pt->buf_row0;
    d.own0 = own0;
    d.own1 = own0 + pt->own_rows;
    // output row y of the buffer goes to row y - own0 of the part's own rows
    d.dst = static_cast<uint8_t *>(pt->dst) - (ptrdiff_t)own0 * (ptrdiff_t)pt->dst_pitch;
    {
        const double nw = (double)pt->p.wiener_w * (double)window_rows(pt->p);
        d.inv_den = 1.0 / (nw * nw * (double)pt->H * (double)pt->W);
    }
    const int ry = window_rows(pt->p) / 2;
    const int TH = t.region_h - 2 * ry;
    d.tiles_y = (pt->own_rows + TH - 1) / TH;
    d.p2_items = 0;
    return d;
}

static hd_status part_launch(const hd_part *pt, void *ws, size_t ws_bytes, int phase, cudaStream_t s)
{
    size_t need = 0;
    hd_status st = hybrid_part_workspace_size(pt, &need);
    if (st != HD_OK) return st;
    if (!ws || ((uintptr_t)ws % kAlign) || ws_bytes < need) return HD_ERR_WORKSPACE;
    const hd_tuning t = current_tuning();
    uint8_t *base = static_cast<uint8_t *>(ws);
    LaunchParams lp;
    std::memset(&lp, 0, sizeof(lp));
    lp.one = part_desc(pt, t, base);
    const int tiles = lp.one.tiles_x * lp.one.tiles_y;
    lp.ticket = reinterpret_cast<unsigned int *>(base);
    lp.ctl_reset = lp.one.ctl;
    lp.ra_max = pt->p.smax / 2;
    lp.wide = image_wide(lp.one);
    if (phase == 1) {
        // the median and statistics tiles; the sums stay in the control block
        lp.oneseg[0] = Seg{0, 1, 0, tiles};
        lp.nsegs = 1;
        lp.total_items = tiles;
        lp.nctl = 0;
    } else {
        // the apply of the own rows from the plane; the last CTA clears the
        // control block for the part's next call
        lp.oneseg[0] = Seg{0, 1, 0, 0};
        lp.nsegs = 1;
        lp.total_items = 0;
        lp.p2_plane = 1;
        lp.nctl = 1;
    }
    int grid = 0;
    size_t smem = 0;
    st = finish_params(lp, t, &grid, &smem);
    if (st != HD_OK) return st;
    if (launch_persistent(lp, grid, smem, (void *)s) != 0) return HD_ERR_CUDA;
    return HD_OK;
}

hd_status hd_part_halo_rows(const hd_params *p, int *rows)
{
    if (!p || !rows) return HD_ERR_ARG;
    if (p->smax < 3 || p->smax > HD_SMAX_MAX || (p->smax & 1) == 0) return HD_ERR_SMAX;
    const int wh = window_rows(*p);
    if (p->wiener_w < 1 || p->wiener_w > HD_WIENER_W_MAX || (p->wiener_w & 1) == 0) return HD_ERR_WINDOW;
    if (wh < 1 || wh > HD_WIENER_W_MAX || (wh & 1) == 0) return HD_ERR_WINDOW;
    *rows = p->smax / 2 + wh / 2;
    return HD_OK;
}

hd_status hybrid_part_workspace_size(const hd_part *pt, size_t *bytes)
{
    if (!bytes) return HD_ERR_ARG;
    hd_status st = check_part(pt, false);
    if (st != HD_OK) return st;
    *bytes = ctl_bytes() + round_up((size_t)pt->buf_rows * f_pitch_of(pt->W, pt->dtype), kAlign) +
             part_plane_bytes(pt);
    return HD_OK;
}

hd_status hybrid_part_stats(const hd_part *pt, void *workspace, size_t ws_bytes, unsigned long long *sums_out,
                            hd_stream_t stream)
{
    hd_status st = check_part(pt, false);
    if (st != HD_OK) return st;
    if (!sums_out || ((uintptr_t)sums_out & 7)) return HD_ERR_ARG;
    size_t need = 0;
    hybrid_part_workspace_size(pt, &need);
    if (!workspace || ((uintptr_t)workspace % kAlign) || ws_bytes < need) return HD_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    // the part's sums start from zero
    if (cudaMemsetAsync(workspace, 0, ctl_bytes(), s) != cudaSuccess) return HD_ERR_CUDA;
    st = part_launch(pt, workspace, ws_bytes, 1, s);
    if (st != HD_OK) return st;
    const ImgCtl *ctl = reinterpret_cast<const ImgCtl *>(static_cast<uint8_t *>(workspace) + kTicketBytes);
    if (cudaMemcpyAsync(sums_out, &ctl->A_lo32, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s) !=
        cudaSuccess)
        return HD_ERR_CUDA;
    return HD_OK;
}

hd_status hybrid_part_apply(const hd_part *pt, const unsigned long long *sums, void *workspace, size_t ws_bytes,
                            hd_stream_t stream)
{
    hd_status st = check_part(pt, true);
    if (st != HD_OK) return st;
    if (!sums || ((uintptr_t)sums & 7)) return HD_ERR_ARG;
    size_t need = 0;
    hybrid_part_workspace_size(pt, &need);
    if (!workspace || ((uintptr_t)workspace % kAlign) || ws_bytes < need) return HD_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    ImgCtl *ctl = reinterpret_cast<ImgCtl *>(static_cast<uint8_t *>(workspace) + kTicketBytes);
    // the whole image's sums replace the part's own
    if (cudaMemcpyAsync(&ctl->A_lo32, sums, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToDevice, s) !=
        cudaSuccess)
        return HD_ERR_CUDA;
    return part_launch(pt, workspace, ws_bytes, 2, s);
}

hd_status hd_set_tuning(const hd_tuning *t)
{
    if (!t) return HD_ERR_ARG;
    if (t->region_h < 16 || t->region_h > 128 || (t->region_h % 8) != 0) return HD_ERR_ARG;
    if (t->ctas_per_sm < 0 || t->ctas_per_sm > 8) return HD_ERR_ARG;
    if (t->plane < 0 || t->plane > 3) return HD_ERR_ARG;
    if (t->small_growth < -1 || t->small_growth > 32) return HD_ERR_ARG;
    if (t->select_lanes != 0 && t->select_lanes != 1 && t->select_lanes != 2 && t->select_lanes != 4 &&
        t->select_lanes != 8)
        return HD_ERR_ARG;
    if (t->batch_lag < 0 || t->batch_lag > 64) return HD_ERR_ARG;
    if (t->batch_order < 0 || t->batch_order > 1) return HD_ERR_ARG;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune = *t;
    return HD_OK;
}

hd_status hd_get_tuning(hd_tuning *t)
{
    if (!t) return HD_ERR_ARG;
    *t = current_tuning();
    return HD_OK;
}

hd_status hd_set_spin_limit(unsigned long long polls)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_spin_limit = polls ? polls : kSpinLimit;
    return HD_OK;
}

hd_status hd_get_device_error(hd_stream_t stream)
{
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return HD_ERR_CUDA;
    unsigned int v = 0, vc = 0;
    if (read_and_clear_device_error(&v) != 0) return HD_ERR_CUDA;
    if (read_and_clear_contrast_error(&vc) != 0) return HD_ERR_CUDA;
    if ((v | vc) & DEVERR_TIMEOUT) return HD_ERR_TIMEOUT;
    return HD_OK;
}

const char *hd_status_str(hd_status s)
{
    switch (s) {
    case HD_OK: return "ok";
    case HD_ERR_ARG: return "invalid argument";
    case HD_ERR_SMAX: return "Smax must be an odd integer in [3, HD_SMAX_MAX]";
    case HD_ERR_WINDOW: return "Wiener window must be an odd integer in [1, HD_WIENER_W_MAX]";
    case HD_ERR_DTYPE: return "unsupported dtype or bit depth";
    case HD_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case HD_ERR_CUDA: return "CUDA runtime error";
    case HD_ERR_TIMEOUT: return "a bounded device-side wait timed out";
    case HD_ERR_OVERFLOW: return "size beyond library limits";
    }
    return "unknown status";
}

int hd_version(void) { return 100; }

}  // extern "C"
