// pr_host.cu -- the C ABI of libpr (include/pr.h): scene upload, per-view
// and batched rasterization, shading, adjoint, graph capture.
//
// Orchestration of one (batched) frame, all on the caller's stream:
//   view table -> tile display boxes -> stage (a) bounds -> stage (b) count
//   -> scan -> scatter -> work items -> stage (c) persistent fragment kernel
//   (one launch per tile size) -> resolve -> [stage (d) shade]
// then one device->host read of the status word.  Bin and item buffers are
// sized from a capacity; if a frame overflows them, the counts it reported
// size the buffers and the frame is run again.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "pr_bound.cuh"
#include "pr_launch.h"

using namespace pr;

namespace {

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;  // sole owner of its allocation
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf()
    {
        if (p)
            cudaFree(p);
    }
    template <class T>
    T *as() const
    {
        return static_cast<T *>(p);
    }
};

// Grows b to hold at least `bytes` (contents are not kept).
cudaError_t ensure(DevBuf &b, size_t bytes)
{
    if (bytes <= b.cap && b.p)
        return cudaSuccess;
    if (b.p) {
        cudaFree(b.p);
        b.p = nullptr;
        b.cap = 0;
    }
    const size_t want = std::max<size_t>(bytes + bytes / 4, 256);
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return e;
    }
    b.cap = want;
    return cudaSuccess;
}

template <class T>
struct PinnedBuf {
    T *p = nullptr;
    size_t cap = 0;
    PinnedBuf() = default;
    PinnedBuf(const PinnedBuf &) = delete;  // sole owner of its allocation
    PinnedBuf &operator=(const PinnedBuf &) = delete;
    ~PinnedBuf()
    {
        if (p)
            cudaFreeHost(p);
    }
    cudaError_t ensure(size_t n)
    {
        if (n <= cap && p)
            return cudaSuccess;
        if (p)
            cudaFreeHost(p);
        p = nullptr;
        cap = 0;
        cudaError_t e = cudaMallocHost((void **)&p, std::max<size_t>(n, 1) * sizeof(T));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e;
        }
        cap = std::max<size_t>(n, 1);
        return cudaSuccess;
    }
};

bool is_device_ptr(const void *p)
{
    if (!p)
        return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

pr_status from_cuda(cudaError_t e)
{
    if (e == cudaSuccess)
        return PR_OK;
    if (e == cudaErrorMemoryAllocation)
        return PR_ERR_OOM;
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver)
        return PR_ERR_NO_CUDA;
    return PR_ERR_CUDA;
}

// On failure: clear the runtime's last error (so the caller's later CUDA
// calls do not see it) and return the mapped status.
#define PR_TRY(expr)                                 \
    do {                                             \
        cudaError_t _e = (expr);                     \
        if (_e != cudaSuccess) {                     \
            cudaGetLastError();                      \
            return from_cuda(_e);                    \
        }                                            \
    } while (0)

constexpr int kDefaultTile = 16;
// frames with more key bytes than this have their keys set back to ~0 by the
// frame's reader instead of cleared at the start of the next frame (L2: 126 MB)
constexpr long long kKeysInL2Bytes = 96ll << 20;
inline bool keys_reset_by_reader(long long npix) { return npix * (long long)sizeof(unsigned long long) > kKeysInL2Bytes; }
constexpr int kDefaultSeg = 256;
constexpr long long kMaxPairs = 0x7FFFFFFFll;  // bin entries per frame: work items hold 32-bit offsets

}  // namespace

// Scratch of one batched frame.
struct pr_workspace {
    DevBuf views, offs, rec, hp, tbox, tile_box, tile_cnt, scan, fill, sums, pairs, items, keys, counters, heads;
    DevBuf hit_entry, hit_tile;  // (triangle, tile) hits of the binning count pass, before the scatter
    DevBuf mip;                  // display step: MIP pyramid of the framebuffer image
    DevBuf disp;                 // batched display step: its view and block tables
    PinnedBuf<char> h_disp;      // ... and their host copy
    cudaEvent_t disp_ev = nullptr;  // recorded after the table copy of the last batched display call
    bool disp_ev_pending = false;
    DevBuf cand, cand_off;         // candidate tiles per triangle; prefix sum over the binned triangles
    DevBuf binned;                 // triangles with candidate tiles (listed by the bound pass)
    DevBuf flag_bits, flag_list;   // pixels flagged for the FP64 re-test (bitmap + list)
    DevBuf loss_part;              // training frames: kLossSlots partial sums of each view's loss
    DevBuf stage;                  // device copies of host-side outputs
    long long cap_pairs = 0, cap_items = 0;
    // leading keys known to hold ~0: every frame's reader (the resolve or the
    // shading) sets the keys it reads back to ~0, so a frame clears only
    // beyond this count (and after a new allocation)
    long long keys_clean_n = 0;
    PinnedBuf<ViewDev> h_views;
    PinnedBuf<long long> h_offs;
    PinnedBuf<Counters> h_cnt;
    pr_stats stats{};
    long long last_T = 0;          // triangles of the last frame (debug bounds)
    static constexpr int kEv = 7;  // stage boundaries of one frame
    cudaEvent_t ev[kEv] = {};
    bool ev_ok = false;
    ~pr_workspace()
    {
        for (int k = 0; k < kEv; ++k)
            if (ev[k])
                cudaEventDestroy(ev[k]);
        if (disp_ev)
            cudaEventDestroy(disp_ev);
    }
    cudaError_t events()
    {
        if (ev_ok)
            return cudaSuccess;
        for (int k = 0; k < kEv; ++k)
            if (!ev[k]) {
                cudaError_t e = cudaEventCreate(&ev[k]);
                if (e != cudaSuccess)
                    return e;
            }
        ev_ok = true;
        return cudaSuccess;
    }
    // the device and pinned buffers a captured graph holds pointers into
    // (a graph has its own view and offset tables, and device outputs only)
    std::vector<const void *> buffer_set() const
    {
        return {rec.p, hp.p, tbox.p, tile_box.p, tile_cnt.p, scan.p, fill.p, sums.p, pairs.p, items.p,
                keys.p, counters.p, heads.p, hit_entry.p, hit_tile.p, cand.p, cand_off.p, binned.p, flag_bits.p,
                flag_list.p, h_cnt.p, loss_part.p};
    }
    // stage times of the last completed frame (events already complete)
    void read_stage_times()
    {
        for (int k = 0; k < 8; ++k)
            stats.stage_ms[k] = 0.f;
        if (!ev_ok)
            return;
        for (int k = 0; k + 1 < kEv; ++k) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev[k], ev[k + 1]) == cudaSuccess)
                stats.stage_ms[k] = ms;
            else
                cudaGetLastError();
        }
    }
};

struct pr_foveation {
    float *lut = nullptr;  // device, n + 1 samples of p
    int n = 0;
};

pr_status pr_foveation_create(const float *p_samples, int32_t n, pr_foveation **out)
{
    if (!p_samples || !out || n < 2 || n > 65536)
        return PR_ERR_INVALID_ARG;
    *out = nullptr;
    if (p_samples[0] != 0.f)
        return PR_ERR_INVALID_ARG;
    for (int k = 1; k <= n; ++k)
        if (!std::isfinite(p_samples[k]) || !(p_samples[k] > p_samples[k - 1]))
            return PR_ERR_INVALID_ARG;
    pr_foveation *f = new (std::nothrow) pr_foveation;
    if (!f)
        return PR_ERR_OOM;
    cudaError_t e = cudaMalloc(&f->lut, sizeof(float) * (n + 1));
    if (e == cudaSuccess)
        e = cudaMemcpy(f->lut, p_samples, sizeof(float) * (n + 1), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (f->lut)
            cudaFree(f->lut);
        delete f;
        return from_cuda(e);
    }
    f->n = n;
    *out = f;
    return PR_OK;
}

namespace pr {
const float *pr_foveation_samples(const pr_foveation *f, int *n)
{
    *n = f->n;
    return f->lut;
}
}  // namespace pr

void pr_foveation_free(pr_foveation *f)
{
    if (f) {
        cudaFree(f->lut);
        delete f;
    }
}

struct pr_scene {
    long long V = 0, T = 0;
    DevBuf vtx;   // 2 V float4: (px, py, pz, vx), (vy, vz, 0, 0)
    DevBuf col;   // V float4: (r, g, b, 0)
    DevBuf tri;   // T int4: (i0, i1, i2, 0)
    DevBuf status;  // one device word: ST_NONFINITE after an update with a non-finite value
    int last_fp64 = 0;  // precision form of the last pr_rasterize (pr_shade follows it)
    DevBuf stage; // host input staging
    DevBuf gstage, ostage;  // adjoint: staged host gradient image / host gradient outputs
    pr_workspace ws;
};

struct pr_graph {
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    pr_workspace *ws = nullptr;
    long long npix = 0;
    bool reader_resets = false;         // the replay's reader sets the keys back to ~0 (and its start clears none)
    bool stage_times = false;           // stage events captured as graph nodes
    DevBuf views, offs;                 // the graph's own view and offset tables
    PinnedBuf<Counters> h_cnt;          // the graph's own copy of its last replay's counters
    std::vector<const void *> buffers;  // the workspace's buffers at capture
};

namespace pr {

// Host-side validation of a view and derivation of its device constants,
// shared by every entry point (the scene's arrays are set by the caller).
pr_status derive_view(const pr_view &in, int tile, int bound, int fp64, ViewDev &v)
{
    if (in.W < 1 || in.H < 1 || in.W > 16384 || in.H > 16384)
        return PR_ERR_INVALID_ARG;
    if (in.mode < PR_CLASSIC || in.mode > PR_BOTH)
        return PR_ERR_INVALID_ARG;
    if (!(in.tan_x > 0.f) || !(in.tan_y > 0.f) || !(in.z_near > 0.f) || !std::isfinite(in.tan_x) ||
        !std::isfinite(in.tan_y) || !std::isfinite(in.z_near))
        return PR_ERR_INVALID_ARG;
    if (!std::isfinite(in.k_a) || !std::isfinite(in.k_d))
        return PR_ERR_INVALID_ARG;
    if (!(in.alpha >= 1.f && in.alpha <= 5.f))
        return PR_ERR_INVALID_ARG;
    if (!(in.d[0] >= 0.f && in.d[1] >= 0.f && in.d[0] + in.d[1] <= 1.f + 1e-6f) ||
        ((in.mode == PR_ROLLING || in.mode == PR_BOTH) && in.d[0] + in.d[1] <= 0.f))
        return PR_ERR_INVALID_ARG;
    if (!(in.fovea[0] >= 0.f && in.fovea[0] <= 1.f && in.fovea[1] >= 0.f && in.fovea[1] <= 1.f))
        return PR_ERR_INVALID_ARG;
    if (tile != 8 && tile != 16 && tile != 32)
        return PR_ERR_INVALID_ARG;
    if (!(in.k_s >= 0.f && std::isfinite(in.k_s)) || (in.k_s > 0.f && !(in.shininess >= 1.f && in.shininess <= 4096.f)))
        return PR_ERR_INVALID_ARG;
    if (bound < PR_BOUND_ZENON || bound > PR_BOUND_TRIVIAL)
        return PR_ERR_INVALID_ARG;
    for (int k = 0; k < 16; ++k)
        if (!std::isfinite(in.pose0[k]) || !std::isfinite(in.pose1[k]))
            return PR_ERR_INVALID_ARG;
    std::memset(&v, 0, sizeof v);
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) {
            v.R0[3 * r + c] = in.pose0[4 * r + c];
            v.R1[3 * r + c] = in.pose1[4 * r + c];
        }
        v.T0[r] = in.pose0[4 * r + 3];
        v.T1[r] = in.pose1[4 * r + 3];
    }
    v.tan_x = in.tan_x;
    v.tan_y = in.tan_y;
    v.z_near = in.z_near;
    v.fx = in.fovea[0];
    v.fy = in.fovea[1];
    v.alpha = in.alpha;
    v.inv_alpha = 1.f / in.alpha;
    if (in.foveation) {
        v.p_lut = in.foveation->lut;
        v.p_n = in.foveation->n;
    }
    v.d0 = in.d[0];
    v.d1 = in.d[1];
    v.t_lo = 0.f;
    v.t_hi = std::min(1.f, in.d[0] + in.d[1]);
    double lw[3] = {in.light_w[0], in.light_w[1], in.light_w[2]};
    double ln = std::sqrt(lw[0] * lw[0] + lw[1] * lw[1] + lw[2] * lw[2]);
    if (!(ln > 0.0) || !std::isfinite(ln))
        return PR_ERR_INVALID_ARG;
    for (int r = 0; r < 3; ++r) {
        double a = 0, b = 0;
        for (int c = 0; c < 3; ++c) {
            a += (double)in.pose0[4 * r + c] * lw[c] / ln;
            b += (double)in.pose1[4 * r + c] * lw[c] / ln;
        }
        v.l0[r] = (float)a;
        v.l1[r] = (float)b;
    }
    v.k_a = in.k_a;
    v.k_d = in.k_d;
    v.k_s = in.k_s;
    v.shininess = in.shininess;
    v.W = in.W;
    v.H = in.H;
    v.mode = in.mode;
    v.S = tile;
    {
        // division by the blocks per row as a multiply (the round-up
        // reciprocal of Granlund and Montgomery, 1994): lb bw_mul / 2^40
        // exceeds lb / bw by lb e / (bw 2^40), e = bw_mul bw - 2^40 < bw; for
        // lb < 2^23 and bw <= 2^11 that is below 2^-6 / bw, less than the
        // 1 / bw from any fraction of lb / bw to the next integer, so the
        // floor is exact
        const unsigned long long bw = (unsigned long long)((in.W + kBlkW - 1) / kBlkW);
        v.bw_mul = ((1ull << 40) + bw - 1) / bw;
    }
    v.tiles_x = (in.W + tile - 1) / tile;
    v.tiles_y = (in.H + tile - 1) / tile;
    v.bound = bound;
    v.fp64 = fp64;
    return PR_OK;
}

}  // namespace pr

namespace {

// Host-side derivation of a view's device constants for a scene.
pr_status make_viewdev(const pr_view &in, const pr_scene *sc, int tile, int bound, int fp64, ViewDev &v)
{
    const pr_status ds = derive_view(in, tile, bound, fp64, v);
    if (ds != PR_OK)
        return ds;
    v.T = (int)sc->T;
    v.V = (int)sc->V;
    v.vtx = sc->vtx.as<float4>();
    v.col4 = sc->col.as<float4>();
    v.tri4 = sc->tri.as<int4>();
    v.scene_status = sc->status.as<unsigned>();
    return PR_OK;
}

pr_params default_params(const pr_params *p)
{
    pr_params d{PR_BOUND_ZENON, kDefaultTile, 0, kDefaultSeg, PR_FOV_SECTOR, 0};
    if (p) {
        d = *p;
        if (d.tile == 0)
            d.tile = kDefaultTile;
        if (d.seg <= 0)
            d.seg = kDefaultSeg;
        d.seg = std::min(d.seg, kMaxSeg);
    }
    return d;
}

struct BatchPlan {
    std::vector<int> order;           // views sorted by tile size
    std::vector<ViewDev> vd;          // in `order`
    std::vector<long long> tri_off, tile_off, pix_off, blk_off;
    long long ttot = 0, ntiles = 0, npix = 0, nblk = 0;
    struct Cls {
        int S;
        bool fp64;
        long long tile_lo, tile_hi;
    };
    bool any_fp64 = false;
    bool any_paper_fov = false;  // some foveated view asks for the paper's edge bound
    bool any_loss = false;       // some view of a training frame accumulates its loss
    std::vector<Cls> classes;
    // output staging: per view (in order) device pointers used by kernels
    std::vector<pr_frame_grad> grads;  // per view (in order); empty: no adjoint
    struct Out {
        uint32_t *id_user;
        float *depth_user, *rgb_user;
        bool id_host, depth_host, rgb_host;
        long long id_off, depth_off, rgb_off;  // byte offsets in ws->stage, -1 = none
    };
    std::vector<Out> out;
    size_t stage_bytes = 0;
};

pr_status plan_batch(const pr_batch_view *views, int n, const pr_params &prm, BatchPlan &P,
                     const pr_frame_grad *grads = nullptr)
{
    if (n < 1 || !views)
        return PR_ERR_INVALID_ARG;
    std::vector<int> tiles(n);
    for (int k = 0; k < n; ++k) {
        tiles[k] = views[k].tile ? views[k].tile : prm.tile;
        if (!views[k].scene)
            return PR_ERR_INVALID_ARG;
    }
    P.order.resize(n);
    for (int k = 0; k < n; ++k)
        P.order[k] = k;
    // views of one tile size and one precision form run in one fragment launch
    std::stable_sort(P.order.begin(), P.order.end(), [&](int a, int b) { return tiles[a] < tiles[b]; });
    P.vd.resize(n);
    P.out.resize(n);
    P.tri_off.assign(n + 1, 0);
    P.tile_off.assign(n + 1, 0);
    P.pix_off.assign(n + 1, 0);
    P.blk_off.assign(n + 1, 0);
    size_t stage = 0;
    auto take = [&](size_t bytes) {
        long long off = (long long)stage;
        stage += (bytes + 255) & ~(size_t)255;
        return off;
    };
    for (int q = 0; q < n; ++q) {
        const pr_batch_view &bv = views[P.order[q]];
        pr_status s = make_viewdev(bv.view, bv.scene, tiles[P.order[q]], prm.bound, prm.fp64_retest, P.vd[q]);
        if (s != PR_OK)
            return s;
        if (prm.fov_bound < PR_FOV_SECTOR || prm.fov_bound > PR_FOV_RECURSIVE)
            return PR_ERR_INVALID_ARG;
        P.vd[q].fov_bound = prm.fov_bound;
        P.any_paper_fov |= prm.fov_bound != PR_FOV_SECTOR && (bv.view.mode == PR_FOVEATED || bv.view.mode == PR_BOTH);
        ViewDev &v = P.vd[q];
        v.tri_off = P.tri_off[q];
        v.tile_off = P.tile_off[q];
        v.pix_off = P.pix_off[q];
        v.blk_off = P.blk_off[q];
        P.blk_off[q + 1] = P.blk_off[q] + pixel_blocks(v.W, v.H);
        P.tri_off[q + 1] = P.tri_off[q] + bv.scene->T;
        P.tile_off[q + 1] = P.tile_off[q] + (long long)v.tiles_x * v.tiles_y;
        P.pix_off[q + 1] = P.pix_off[q] + (long long)v.W * v.H;
        const long long np = (long long)v.W * v.H;
        BatchPlan::Out &o = P.out[q];
        o.id_user = bv.id_out;
        o.depth_user = bv.depth_out;
        o.rgb_user = bv.rgb_out;
        o.id_host = bv.id_out && !is_device_ptr(bv.id_out);
        o.depth_host = bv.depth_out && !is_device_ptr(bv.depth_out);
        o.rgb_host = bv.rgb_out && !is_device_ptr(bv.rgb_out);
        // ids are staged when the caller's buffer is on the host or absent
        // but shading needs them
        o.id_off = (o.id_host || (!bv.id_out && bv.rgb_out)) ? take(np * 4) : -1;
        o.depth_off = o.depth_host ? take(np * 4) : -1;
        o.rgb_off = o.rgb_host ? take(np * 12) : -1;
    }
    if (grads) {
        P.grads.resize(n);
        for (int q = 0; q < n; ++q) {
            const pr_frame_grad &g = grads[P.order[q]];
            const pr_batch_view &bv = views[P.order[q]];
            const int nsrc = (g.grad_rgb != nullptr) + (g.target_rgb != nullptr) + (g.target_u8 != nullptr);
            if (nsrc > 1 || (g.loss && !g.target_rgb && !g.target_u8))
                return PR_ERR_INVALID_ARG;  // one gradient source; a loss needs a target
            if (nsrc && (P.out[q].rgb_host || (g.grad_rgb && !is_device_ptr(g.grad_rgb)) ||
                         (g.target_rgb && !is_device_ptr(g.target_rgb)) ||
                         (g.target_u8 && !is_device_ptr(g.target_u8)) || (g.loss && !is_device_ptr(g.loss)) ||
                         (g.dcol && !is_device_ptr(g.dcol)) || (g.dpos && !is_device_ptr(g.dpos)) ||
                         (g.dvel && !is_device_ptr(g.dvel))))
                return PR_ERR_INVALID_ARG;  // the adjoint in a frame needs device buffers
            P.grads[q] = g;
            P.any_loss |= g.loss != nullptr;
        }
    }
    P.ttot = P.tri_off[n];
    P.ntiles = P.tile_off[n];
    P.npix = P.pix_off[n];
    P.nblk = P.blk_off[n];
    P.stage_bytes = stage;
    if (P.ttot >= (1ll << 32) - 1)
        return PR_ERR_INVALID_ARG;
    for (int q = 0; q < n; ++q) {
        const int S = P.vd[q].S;
        const bool f = P.vd[q].fp64 != 0;
        P.any_fp64 |= f;
        if (P.classes.empty() || P.classes.back().S != S || P.classes.back().fp64 != f)
            P.classes.push_back({S, f, P.tile_off[q], P.tile_off[q + 1]});
        else
            P.classes.back().tile_hi = P.tile_off[q + 1];
    }
    return PR_OK;
}

// Sizes every buffer of the workspace for the plan (eager calls only).
pr_status size_workspace(pr_workspace *ws, const BatchPlan &P, int seg)
{
    const int n = (int)P.vd.size();
    PR_TRY(ensure(ws->views, sizeof(ViewDev) * n));
    PR_TRY(ensure(ws->offs, sizeof(long long) * 4 * (n + 1)));
    PR_TRY(ensure(ws->rec, sizeof(float4) * kRecF4 * std::max(P.ttot, 1ll)));
    PR_TRY(ensure(ws->hp, sizeof(float4) * kMaxHp * std::max(P.ttot, 1ll)));
    PR_TRY(ensure(ws->tbox, sizeof(int4) * std::max(P.ttot, 1ll)));
    PR_TRY(ensure(ws->tile_box, sizeof(float4) * std::max(P.ntiles, 1ll)));
    PR_TRY(ensure(ws->tile_cnt, sizeof(unsigned long long) * std::max(P.ntiles, 1ll)));
    PR_TRY(ensure(ws->scan, sizeof(unsigned long long) * (P.ntiles + 1)));
    PR_TRY(ensure(ws->fill, sizeof(unsigned) * std::max(P.ntiles, 1ll)));
    // two scans' look-back states: the candidate-tile scan, then the tile scan
    PR_TRY(ensure(ws->sums,
                  sizeof(unsigned long long) * (scan_block_sums_needed(P.ttot) + scan_block_sums_needed(P.ntiles))));
    PR_TRY(ensure(ws->cand, sizeof(unsigned long long) * std::max(P.ttot, 1ll)));
    PR_TRY(ensure(ws->cand_off, sizeof(unsigned long long) * (P.ttot + 1)));
    PR_TRY(ensure(ws->binned, sizeof(int) * std::max(P.ttot, 1ll)));
    const void *old_keys = ws->keys.p;
    PR_TRY(ensure(ws->keys, sizeof(unsigned long long) * std::max(P.npix, 1ll)));
    if (ws->keys.p != old_keys)
        ws->keys_clean_n = 0;
    if (P.any_loss)
        PR_TRY(ensure(ws->loss_part, sizeof(float) * kLossSlots * n));
    if (P.any_fp64) {
        PR_TRY(ensure(ws->flag_bits, sizeof(unsigned) * ((P.npix + 31) / 32 + 1)));
        PR_TRY(ensure(ws->flag_list, sizeof(long long) * std::max(P.npix, 1ll)));
    }
    PR_TRY(ensure(ws->counters, sizeof(Counters)));
    PR_TRY(ensure(ws->heads, sizeof(int) * 8));
    PR_TRY(ensure(ws->stage, std::max<size_t>(P.stage_bytes, 256)));
    const long long want_pairs = std::min(std::max(ws->cap_pairs, 2 * P.ttot + P.ntiles + 1024), kMaxPairs);
    if ((size_t)want_pairs * sizeof(unsigned long long) > ws->pairs.cap || !ws->pairs.p) {
        PR_TRY(ensure(ws->pairs, sizeof(unsigned long long) * want_pairs));
    }
    ws->cap_pairs = std::min((long long)(ws->pairs.cap / sizeof(unsigned long long)), kMaxPairs);
    PR_TRY(ensure(ws->hit_entry, sizeof(unsigned long long) * ws->cap_pairs));
    PR_TRY(ensure(ws->hit_tile, sizeof(unsigned) * ws->cap_pairs));
    const long long want_items = std::max(ws->cap_items, ws->cap_pairs / seg + P.ntiles + 1024);
    if ((size_t)want_items * sizeof(int4) > ws->items.cap || !ws->items.p) {
        PR_TRY(ensure(ws->items, sizeof(int4) * want_items));
    }
    ws->cap_items = std::min((long long)(ws->items.cap / sizeof(int4)), kMaxPairs);
    PR_TRY(ws->h_views.ensure(n));
    PR_TRY(ws->h_offs.ensure(4 * (n + 1)));
    PR_TRY(ws->h_cnt.ensure(1));
    return PR_OK;
}

// Writes the frame's view and offset tables into the workspace's pinned
// host copies (h_views: n views; h_offs: triangle, tile, pixel and warp
// block offsets, n + 1 each).  shade: views with an rgb output get one.
void fill_tables(pr_workspace *ws, BatchPlan &P, bool shade)
{
    const int n = (int)P.vd.size();
    char *stage = ws->stage.as<char>();
    for (int q = 0; q < n; ++q) {
        ViewDev &v = P.vd[q];
        const BatchPlan::Out &o = P.out[q];
        v.id_out = o.id_off >= 0 ? (uint32_t *)(stage + o.id_off) : o.id_user;
        v.depth_out = o.depth_off >= 0 ? (float *)(stage + o.depth_off) : o.depth_user;
        v.id_in = v.id_out;
        v.rgb_out = shade ? (o.rgb_off >= 0 ? (float *)(stage + o.rgb_off) : o.rgb_user) : nullptr;
        v.rec = ws->rec.as<float4>();  // shading in the same frame reads its records
        if (!P.grads.empty()) {
            const pr_frame_grad &g = P.grads[q];
            v.grad_in = g.grad_rgb;
            v.target = g.target_rgb;
            v.target_u8 = g.target_u8;
            v.loss = (g.target_rgb || g.target_u8) ? g.loss : nullptr;
            v.loss_part = v.loss ? ws->loss_part.as<float>() + (size_t)kLossSlots * q : nullptr;
            v.dcol = g.dcol;
            v.dpos = g.dpos;
            v.dvel = g.dvel;
        }
        ws->h_views.p[q] = v;
    }
    long long *ho = ws->h_offs.p;
    for (int q = 0; q <= n; ++q) {
        ho[q] = P.tri_off[q];
        ho[n + 1 + q] = P.tile_off[q];
        ho[2 * (n + 1) + q] = P.pix_off[q];
        ho[3 * (n + 1) + q] = P.blk_off[q];
    }
}

// Enqueues one frame (no host synchronisation).  shade: also run stage (d)
// for views with an rgb output.  tables: device view and offset tables that
// already hold what fill_tables wrote (a captured graph's own copies), or
// null to upload the workspace's tables in the same sequence.  marks: record
// the stage events (always when not capturing).
pr_status enqueue_batch(pr_workspace *ws, BatchPlan &P, int seg, bool shade, cudaStream_t st,
                        const ViewDev *tab_views = nullptr, const long long *tab_offs = nullptr, bool marks = true,
                        Counters *h_cnt = nullptr)
{
    const int n = (int)P.vd.size();
    char *stage = ws->stage.as<char>();
    if (!tab_views) {
        fill_tables(ws, P, shade);
        PR_TRY(cudaMemcpyAsync(ws->views.p, ws->h_views.p, sizeof(ViewDev) * n, cudaMemcpyHostToDevice, st));
        PR_TRY(cudaMemcpyAsync(ws->offs.p, ws->h_offs.p, sizeof(long long) * 4 * (n + 1), cudaMemcpyHostToDevice, st));
        tab_views = ws->views.as<ViewDev>();
        tab_offs = ws->offs.as<long long>();
    }
    const ViewDev *dv = tab_views;
    const long long *tri_offs = tab_offs, *tile_offs = tri_offs + n + 1, *pix_offs = tile_offs + n + 1;
    const long long *blk_offs = pix_offs + n + 1;
    Counters *cnt = ws->counters.as<Counters>();
    unsigned long long *state_a = ws->sums.as<unsigned long long>();
    unsigned long long *state_b = state_a + scan_block_sums_needed(P.ttot);
    float4 *rec = ws->rec.as<float4>(), *hp = ws->hp.as<float4>(), *tile_box = ws->tile_box.as<float4>();
    int4 *tbox = ws->tbox.as<int4>();
    unsigned long long *tile_cnt = ws->tile_cnt.as<unsigned long long>(), *scan = ws->scan.as<unsigned long long>();
    PR_TRY(ws->events());
    cudaEvent_t *ev = ws->ev;
    // while capturing, external records keep the events as graph nodes
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    PR_TRY(cudaStreamIsCapturing(st, &cs));
    const bool capturing = cs == cudaStreamCaptureStatusActive;
    const unsigned ev_flags = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    auto mark = [&](int k) {
        return marks || !capturing ? cudaEventRecordWithFlags(ev[k], st, ev_flags) : cudaSuccess;
    };
    unsigned long long *cand = ws->cand.as<unsigned long long>(), *cand_off = ws->cand_off.as<unsigned long long>();
    PR_TRY(mark(0));
    // one launch clears the counters, queue heads, tile counts and cursors,
    // both scans' tickets and flags, the FP64 flags, and computes the tiles'
    // display boxes.  The keys: a frame whose keys fit in L2 clears them
    // here, where the fragment stage then finds them in L2; a larger frame
    // has its reader (resolve or shading, which reads every key anyway) set
    // them back to ~0 for the next frame, and clears here only the keys that
    // earlier frames' readers have not left so (the state is unknown until
    // this frame's reader is enqueued)
    const bool reader_resets = keys_reset_by_reader(P.npix);
    const long long clean_before = reader_resets ? ws->keys_clean_n : 0;
    ws->keys_clean_n = 0;
    PR_TRY(launch_frame_init(dv, n, tile_offs, tile_box, cnt, ws->heads.as<int>(), tile_cnt, ws->fill.as<unsigned>(),
                             P.ntiles, state_a, scan_state_words(P.ttot), state_b, scan_state_words(P.ntiles),
                             ws->flag_bits.as<unsigned>(), P.any_fp64 ? (P.npix + 31) / 32 + 1 : 0,
                             ws->keys.as<unsigned long long>(), P.npix > clean_before ? P.npix : 0,
                             ws->loss_part.as<float>(), P.any_loss ? (long long)kLossSlots * n : 0, st));
    int *binned = ws->binned.as<int>();
    PR_TRY(launch_bound(dv, n, tri_offs, P.ttot, rec, hp, tbox, cand, binned, cnt, st));
    if (P.any_paper_fov)
        PR_TRY(launch_paper_fov(dv, n, tri_offs, P.ttot, rec, hp, tbox, cand, st));
    PR_TRY(mark(1));
    // candidate tiles of the binned triangles (count known on the device)
    PR_TRY(launch_scan(cand, cand_off, state_a, P.ttot, 0, cnt, st, true, binned, &cnt->binned));
    PR_TRY(launch_bin_count(dv, n, tri_offs, P.ttot, binned, cand_off, rec, hp, tbox, tile_box, tile_cnt,
                            ws->hit_entry.as<unsigned long long>(), ws->hit_tile.as<unsigned>(), ws->cap_pairs, cnt,
                            st));
    // the scan of the tile counts also emits the work items
    ItemsOut io;
    io.views = dv;
    io.nviews = n;
    io.tile_offs = tile_offs;
    io.items = ws->items.as<int4>();
    io.cap_items = ws->cap_items;
    io.cap_pairs = ws->cap_pairs;
    PR_TRY(launch_scan(tile_cnt, scan, state_b, P.ntiles, seg, cnt, st, true, nullptr, nullptr, &io));
    PR_TRY(launch_bin_scatter(ws->hit_entry.as<unsigned long long>(), ws->hit_tile.as<unsigned>(), scan,
                              ws->fill.as<unsigned>(), ws->pairs.as<unsigned long long>(), ws->cap_pairs, P.ntiles, cnt,
                              st));
    PR_TRY(launch_sort_items(ws->items.as<int4>(), scan, P.ntiles, ws->cap_items, seg,
                             ws->pairs.as<unsigned long long>(), cnt, st));
    PR_TRY(mark(2));
    int *heads = ws->heads.as<int>();
    for (size_t c = 0; c < P.classes.size(); ++c) {
        const auto &cl = P.classes[c];
        PR_TRY(launch_fragment(cl.S, cl.fp64, dv, ws->items.as<int4>(), scan, cl.tile_lo, cl.tile_hi, ws->cap_items,
                               heads + c, ws->pairs.as<unsigned long long>(), rec, ws->keys.as<unsigned long long>(),
                               ws->flag_bits.as<unsigned>(), ws->flag_list.as<long long>(), cnt,
                               fragment_grid(cl.S, cl.fp64), st));
    }
    PR_TRY(mark(3));
    if (P.any_fp64)
        PR_TRY(launch_retest(dv, n, pix_offs, scan, tile_cnt, ws->pairs.as<unsigned long long>(), rec,
                             ws->flag_list.as<long long>(), ws->keys.as<unsigned long long>(), ws->cap_pairs, cnt, st));
    PR_TRY(mark(4));
    if (!shade)
        PR_TRY(launch_resolve(dv, n, pix_offs, P.npix, ws->keys.as<unsigned long long>(), reader_resets, st));
    PR_TRY(mark(5));
    if (shade)  // resolves the keys too, and in a training frame runs the adjoint
        PR_TRY(launch_shade(dv, n, blk_offs, P.nblk, ws->keys.as<unsigned long long>(), reader_resets,
                            !P.grads.empty(), cnt, shade_features(P.vd.data(), n), st, P.vd.data()));
    if (shade && P.any_loss)  // the views' loss partial sums into the callers' losses
        PR_TRY(launch_loss_finalize(dv, n, cnt, st));
    // the reader has set every key of the frame back to ~0
    if (reader_resets)
        ws->keys_clean_n = std::max(clean_before, P.npix);
    PR_TRY(mark(6));
    // host-side outputs
    for (int q = 0; q < n; ++q) {
        const BatchPlan::Out &o = P.out[q];
        const long long np = (long long)P.vd[q].W * P.vd[q].H;
        if (o.id_host)
            PR_TRY(cudaMemcpyAsync(o.id_user, stage + o.id_off, np * 4, cudaMemcpyDeviceToHost, st));
        if (o.depth_host)
            PR_TRY(cudaMemcpyAsync(o.depth_user, stage + o.depth_off, np * 4, cudaMemcpyDeviceToHost, st));
        if (shade && o.rgb_host)
            PR_TRY(cudaMemcpyAsync(o.rgb_user, stage + o.rgb_off, np * 12, cudaMemcpyDeviceToHost, st));
    }
    // the frame's counters to the host: the workspace's copy, or the graph's
    // own (so a replay's status can be read while the next replay runs)
    PR_TRY(cudaMemcpyAsync(h_cnt ? h_cnt : ws->h_cnt.p, ws->counters.p, sizeof(Counters), cudaMemcpyDeviceToHost,
                           st));
    return PR_OK;
}

pr_status finish_stats(pr_workspace *ws, const BatchPlan &P)
{
    const Counters &c = *ws->h_cnt.p;
    ws->stats.tests = c.tests;
    ws->stats.hits = c.hits;
    ws->stats.pairs = c.pairs_total;
    ws->stats.items = c.items_total;
    ws->stats.culled = c.culled;
    ws->stats.flagged = c.flagged;
    ws->stats.changed = c.changed;
    {
        unsigned b = c.depth_err_bits;
        float e;
        std::memcpy(&e, &b, sizeof e);
        ws->stats.fp64_depth_err = e;
    }
    ws->stats.pixels = (uint64_t)P.npix;
    ws->last_T = P.ttot;
    ws->read_stage_times();
    if (c.status & ST_TIMEOUT)
        return PR_ERR_TIMEOUT;
    if (c.status & ST_NONFINITE)
        return PR_ERR_NONFINITE;  // a scene updated with a non-finite value: its triangles were culled
    if (c.status & ST_BAD_INDEX)
        return PR_ERR_CUDA;  // a kernel's own bounds check caught an inconsistent index (and skipped it)
    if (c.status & (ST_OVERFLOW_PAIRS | ST_OVERFLOW_ITEMS | ST_OVERFLOW_FLAGS))
        return PR_ERR_OVERFLOW;
    return PR_OK;
}

// Eager frame: enqueue, read the status, regrow and rerun on overflow.
pr_status run_batch(pr_workspace *ws, const pr_batch_view *views, int n, const pr_params *params, bool shade,
                    cudaStream_t st, const pr_frame_grad *grads = nullptr)
{
    pr_params prm = default_params(params);
    BatchPlan P;
    pr_status s = plan_batch(views, n, prm, P, grads);
    if (s != PR_OK)
        return s;
    for (int attempt = 0; attempt < 3; ++attempt) {
        s = size_workspace(ws, P, prm.seg);
        if (s != PR_OK)
            return s;
        s = enqueue_batch(ws, P, prm.seg, shade, st);
        if (s != PR_OK)
            return s;
        PR_TRY(cudaStreamSynchronize(st));
        s = finish_stats(ws, P);
        if (s != PR_ERR_OVERFLOW)
            return s;
        const Counters &c = *ws->h_cnt.p;
        // work items address bin entries with 32-bit offsets: a frame with
        // more entries than that is refused, not regrown
        if ((long long)c.pairs_total > kMaxPairs || (long long)c.items_total > kMaxPairs)
            return PR_ERR_OVERFLOW;
        ws->cap_pairs = std::max<long long>(ws->cap_pairs, (long long)c.pairs_total + 1024);
        ws->cap_items = std::max<long long>(ws->cap_items, (long long)c.items_total + 1024);
        ws->cap_pairs = std::min(ws->cap_pairs + ws->cap_pairs / 4, kMaxPairs);
        ws->cap_items = std::min(ws->cap_items + ws->cap_items / 4, kMaxPairs);  // size_workspace grows both to these
    }
    return PR_ERR_OVERFLOW;
}

pr_status single_view(pr_scene *sc, const pr_view *view, const pr_params *params, uint32_t *id_out,
                      float *depth_out, float *rgb_out, cudaStream_t st)
{
    if (!sc || !view)
        return PR_ERR_INVALID_ARG;
    pr_batch_view bv;
    std::memset(&bv, 0, sizeof bv);
    bv.scene = sc;
    bv.view = *view;
    bv.id_out = id_out;
    bv.depth_out = depth_out;
    bv.rgb_out = rgb_out;
    return run_batch(&sc->ws, &bv, 1, params, rgb_out != nullptr, st);
}

// One-view table for stages (d)/(e) called on their own.
pr_status upload_single(pr_scene *sc, const ViewDev &v, cudaStream_t st)
{
    pr_workspace *ws = &sc->ws;
    PR_TRY(ensure(ws->views, sizeof(ViewDev)));
    PR_TRY(ensure(ws->offs, sizeof(long long) * 6));
    PR_TRY(ws->h_views.ensure(1));
    PR_TRY(ws->h_offs.ensure(6));
    ws->h_views.p[0] = v;
    long long *o = ws->h_offs.p;
    o[0] = 0;
    o[1] = pixel_blocks(v.W, v.H);  // warp pixel blocks
    o[2] = o[3] = o[4] = o[5] = 0;
    PR_TRY(cudaMemcpyAsync(ws->views.p, ws->h_views.p, sizeof(ViewDev), cudaMemcpyHostToDevice, st));
    PR_TRY(cudaMemcpyAsync(ws->offs.p, o, sizeof(long long) * 2, cudaMemcpyHostToDevice, st));
    return PR_OK;
}

}  // namespace

// =============================================================== C ABI

extern "C" {

int32_t pr_version(void) { return 1; }

pr_status pr_debug_scan_timeout(void *stream)
{
    unsigned status = 0u;
    PR_TRY(scan_timeout_probe((cudaStream_t)stream, &status));
    return (status & ST_TIMEOUT) ? PR_ERR_TIMEOUT : PR_OK;
}

pr_status pr_measure_fp32_peak(void *stream, double *tflops_out)
{
    if (!tflops_out)
        return PR_ERR_INVALID_ARG;
    *tflops_out = 0.0;
    PR_TRY(measure_fma_peak((cudaStream_t)stream, tflops_out));
    return PR_OK;
}

const char *pr_status_string(pr_status s)
{
    switch (s) {
    case PR_OK: return "ok";
    case PR_ERR_INVALID_ARG: return "invalid argument";
    case PR_ERR_CUDA: return "CUDA error";
    case PR_ERR_OOM: return "out of device memory";
    case PR_ERR_OVERFLOW: return "device buffer overflow";
    case PR_ERR_TIMEOUT: return "device wait timed out";
    case PR_ERR_NONFINITE: return "non-finite input";
    case PR_ERR_NO_CUDA: return "no CUDA device";
    }
    return "unknown status";
}

static pr_status copy_in(const void *src, size_t bytes, DevBuf &stage, const void **dev, cudaStream_t st)
{
    if (is_device_ptr(src)) {
        *dev = src;
        return PR_OK;
    }
    PR_TRY(ensure(stage, bytes));
    PR_TRY(cudaMemcpyAsync(stage.p, src, bytes, cudaMemcpyHostToDevice, st));
    *dev = stage.p;
    return PR_OK;
}

static pr_status check_scene_status(pr_scene *sc, cudaStream_t st)
{
    pr_workspace *ws = &sc->ws;
    PR_TRY(ws->h_cnt.ensure(1));
    PR_TRY(cudaMemcpyAsync(ws->h_cnt.p, ws->counters.p, sizeof(Counters), cudaMemcpyDeviceToHost, st));
    PR_TRY(cudaStreamSynchronize(st));
    const unsigned s = ws->h_cnt.p->status;
    if (s & ST_NONFINITE)
        return PR_ERR_NONFINITE;
    if (s & ST_BAD_INDEX)
        return PR_ERR_INVALID_ARG;
    return PR_OK;
}

pr_status pr_scene_update(pr_scene *sc, const float *pos, const float *vel, const float *col, void *stream)
{
    if (!sc)
        return PR_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    const long long V = sc->V;
    PR_TRY(cudaMemsetAsync(sc->status.p, 0, sizeof(unsigned), st));
    // write each given [V][3] array into the vertex records / colours
    const float *arrs[3] = {pos, vel, col};
    for (int a = 0; a < 3; ++a) {
        if (!arrs[a])
            continue;
        const void *d = nullptr;
        pr_status s = copy_in(arrs[a], sizeof(float) * 3 * V, sc->stage, &d, st);
        if (s != PR_OK)
            return s;
        PR_TRY(launch_scene_set((const float *)d, a, V, sc->vtx.as<float4>(), sc->col.as<float4>(), st));
    }
    // a non-finite value is reported by the next frame that reads the scene
    PR_TRY(launch_scene_check(sc->vtx.as<float4>(), sc->col.as<float4>(), V, sc->status.as<unsigned>(), st));
    return PR_OK;
}

pr_status pr_scene_update_batch(pr_scene *const *scenes, int32_t n, const float *const *pos,
                                const float *const *vel, const float *const *col, void *stream)
{
    if (!scenes || n < 1 || n > 4096)
        return PR_ERR_INVALID_ARG;
    std::vector<SceneUpdate> u((size_t)n);
    for (int k = 0; k < n; ++k) {
        pr_scene *sc = scenes[k];
        if (!sc)
            return PR_ERR_INVALID_ARG;
        const float *p = pos ? pos[k] : nullptr, *w = vel ? vel[k] : nullptr, *c = col ? col[k] : nullptr;
        if ((p && !is_device_ptr(p)) || (w && !is_device_ptr(w)) || (c && !is_device_ptr(c)))
            return PR_ERR_INVALID_ARG;  // device arrays only (no staging)
        u[k] = SceneUpdate{sc->vtx.as<float4>(), sc->col.as<float4>(), sc->status.as<unsigned>(), p, w, c, sc->V};
    }
    PR_TRY(launch_scene_update_batch(u.data(), n, (cudaStream_t)stream));
    return PR_OK;
}

pr_status pr_scene_upload(const float *pos, const float *vel, const float *col, const int32_t *tri, int64_t V,
                          int64_t T, void *stream, pr_scene **out)
{
    if (!out || !pos || !vel || !col || (T > 0 && !tri) || V < 1 || T < 0 || V > (1ll << 30) || T > (1ll << 30))
        return PR_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return PR_ERR_NO_CUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    pr_scene *sc = new (std::nothrow) pr_scene;
    if (!sc)
        return PR_ERR_OOM;
    sc->V = V;
    sc->T = T;
    pr_status s = from_cuda(ensure(sc->vtx, sizeof(float4) * 2 * V));
    if (s == PR_OK)
        s = from_cuda(ensure(sc->col, sizeof(float4) * V));
    if (s == PR_OK)
        s = from_cuda(ensure(sc->tri, sizeof(int4) * std::max<int64_t>(T, 1)));
    if (s == PR_OK)
        s = from_cuda(ensure(sc->ws.counters, sizeof(Counters)));
    if (s == PR_OK)
        s = from_cuda(ensure(sc->status, sizeof(unsigned)));
    if (s == PR_OK)
        s = from_cuda(cudaMemsetAsync(sc->ws.counters.p, 0, sizeof(Counters), st));
    if (s == PR_OK)
        s = from_cuda(cudaMemsetAsync(sc->status.p, 0, sizeof(unsigned), st));
    // stage the three [V][3] arrays and the index array
    DevBuf sp, sv, scol, stri;
    const void *dp = nullptr, *dvel = nullptr, *dc = nullptr, *dt = nullptr;
    if (s == PR_OK)
        s = copy_in(pos, sizeof(float) * 3 * V, sp, &dp, st);
    if (s == PR_OK)
        s = copy_in(vel, sizeof(float) * 3 * V, sv, &dvel, st);
    if (s == PR_OK)
        s = copy_in(col, sizeof(float) * 3 * V, scol, &dc, st);
    if (s == PR_OK && T > 0)
        s = copy_in(tri, sizeof(int) * 3 * T, stri, &dt, st);
    if (s == PR_OK)
        s = from_cuda(launch_scene_pack((const float *)dp, (const float *)dvel, (const float *)dc, V,
                                        sc->vtx.as<float4>(), sc->col.as<float4>(), st));
    if (s == PR_OK && T > 0)
        s = from_cuda(launch_scene_idx((const int *)dt, T, V, sc->tri.as<int4>(), sc->ws.counters.as<Counters>(), st));
    if (s == PR_OK)
        s = from_cuda(launch_scene_check(sc->vtx.as<float4>(), sc->col.as<float4>(), V,
                                         &sc->ws.counters.as<Counters>()->status, st));
    if (s == PR_OK)
        s = check_scene_status(sc, st);  // synchronises: staging buffers may be released
    if (s != PR_OK) {
        cudaStreamSynchronize(st);
        delete sc;
        return s;
    }
    *out = sc;
    return PR_OK;
}

void pr_scene_free(pr_scene *sc)
{
    if (sc) {
        cudaDeviceSynchronize();
        delete sc;
    }
}

pr_status pr_rasterize(pr_scene *sc, const pr_view *view, const pr_params *params, uint32_t *id_out, float *depth_out,
                       void *stream)
{
    const pr_status s = single_view(sc, view, params, id_out, depth_out, nullptr, (cudaStream_t)stream);
    if (sc)
        sc->last_fp64 = params && params->fp64_retest ? 1 : 0;
    return s;
}

static pr_status stage_in_ids(pr_scene *sc, const uint32_t *id, long long np, const uint32_t **dev, cudaStream_t st)
{
    return copy_in(id, sizeof(uint32_t) * np, sc->stage, (const void **)dev, st);
}

pr_status pr_shade(pr_scene *sc, const pr_view *view, const uint32_t *id, float *rgb_out, void *stream)
{
    if (!sc || !view || !id || !rgb_out)
        return PR_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    ViewDev v;
    pr_status s = make_viewdev(*view, sc, kDefaultTile, PR_BOUND_ZENON, sc->last_fp64, v);
    if (s != PR_OK)
        return s;
    const long long np = (long long)view->W * view->H;
    const uint32_t *did = nullptr;
    s = stage_in_ids(sc, id, np, &did, st);
    if (s != PR_OK)
        return s;
    const bool host_out = !is_device_ptr(rgb_out);
    DevBuf *ob = &sc->ws.stage;
    if (host_out)
        PR_TRY(ensure(*ob, sizeof(float) * 3 * np));
    v.id_in = did;
    v.rgb_out = host_out ? ob->as<float>() : rgb_out;
    s = upload_single(sc, v, st);
    if (s != PR_OK)
        return s;
    PR_TRY(launch_shade(sc->ws.views.as<ViewDev>(), 1, sc->ws.offs.as<long long>(),
                        pixel_blocks(v.W, v.H), nullptr, false, false, nullptr,
                        shade_features(&v, 1), st, &v));
    if (host_out)
        PR_TRY(cudaMemcpyAsync(rgb_out, ob->p, sizeof(float) * 3 * np, cudaMemcpyDeviceToHost, st));
    PR_TRY(cudaStreamSynchronize(st));
    return PR_OK;
}

pr_status pr_backward(pr_scene *sc, const pr_view *view, const uint32_t *id, const float *grad_rgb, float *dcol,
                      float *dpos, float *dvel, void *stream)
{
    if (!sc || !view || !id || !grad_rgb)
        return PR_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    ViewDev v;
    pr_status s = make_viewdev(*view, sc, kDefaultTile, PR_BOUND_ZENON, 0, v);
    if (s != PR_OK)
        return s;
    const long long np = (long long)view->W * view->H;
    const long long V = sc->V;
    // inputs: ids and gradient (staged if on the host)
    const uint32_t *did = nullptr;
    const void *dg = nullptr;
    s = stage_in_ids(sc, id, np, &did, st);
    if (s == PR_OK)
        s = copy_in(grad_rgb, sizeof(float) * 3 * np, sc->gstage, &dg, st);
    if (s != PR_OK)
        return s;
    // outputs: accumulate in place when on the device, else through staging
    float *outs[3] = {dcol, dpos, dvel};
    float *douts[3] = {nullptr, nullptr, nullptr};
    bool host[3] = {false, false, false};
    for (int a = 0; a < 3; ++a) {
        if (!outs[a])
            continue;
        host[a] = !is_device_ptr(outs[a]);
        if (host[a]) {
            PR_TRY(ensure(sc->ostage, sizeof(float) * 9 * V));
            douts[a] = sc->ostage.as<float>() + 3 * a * V;
            PR_TRY(cudaMemcpyAsync(douts[a], outs[a], sizeof(float) * 3 * V, cudaMemcpyHostToDevice, st));
        } else {
            douts[a] = outs[a];
        }
    }
    v.id_in = did;
    v.grad_in = (const float *)dg;
    v.dcol = douts[0];
    v.dpos = douts[1];
    v.dvel = douts[2];
    s = upload_single(sc, v, st);
    if (s != PR_OK)
        return s;
    PR_TRY(launch_backward(sc->ws.views.as<ViewDev>(), 1, sc->ws.offs.as<long long>(),
                           pixel_blocks(v.W, v.H), nullptr, shade_features(&v, 1), st, &v));
    for (int a = 0; a < 3; ++a)
        if (host[a])
            PR_TRY(cudaMemcpyAsync(outs[a], douts[a], sizeof(float) * 3 * V, cudaMemcpyDeviceToHost, st));
    PR_TRY(cudaStreamSynchronize(st));
    return PR_OK;
}

pr_status pr_backward_batch(pr_workspace *ws, const pr_backward_view *views, int32_t n, void *stream)
{
    if (!ws || !views || n < 1)
        return PR_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    PR_TRY(ws->h_views.ensure(n));
    PR_TRY(ws->h_offs.ensure(n + 1));
    PR_TRY(ensure(ws->views, sizeof(ViewDev) * n));
    PR_TRY(ensure(ws->offs, sizeof(long long) * (n + 1)));
    long long *blk = ws->h_offs.p;
    blk[0] = 0;
    for (int k = 0; k < n; ++k) {
        const pr_backward_view &b = views[k];
        if (!b.scene || !b.id || !b.grad_rgb || !is_device_ptr(b.id) || !is_device_ptr(b.grad_rgb) ||
            (b.dcol && !is_device_ptr(b.dcol)) || (b.dpos && !is_device_ptr(b.dpos)) ||
            (b.dvel && !is_device_ptr(b.dvel)))
            return PR_ERR_INVALID_ARG;
        ViewDev v;
        pr_status s = make_viewdev(b.view, b.scene, kDefaultTile, PR_BOUND_ZENON, 0, v);
        if (s != PR_OK)
            return s;
        v.id_in = b.id;
        v.grad_in = b.grad_rgb;
        v.dcol = b.dcol;
        v.dpos = b.dpos;
        v.dvel = b.dvel;
        v.blk_off = blk[k];
        blk[k + 1] = blk[k] + pixel_blocks(v.W, v.H);
        ws->h_views.p[k] = v;
    }
    PR_TRY(cudaMemcpyAsync(ws->views.p, ws->h_views.p, sizeof(ViewDev) * n, cudaMemcpyHostToDevice, st));
    PR_TRY(cudaMemcpyAsync(ws->offs.p, blk, sizeof(long long) * (n + 1), cudaMemcpyHostToDevice, st));
    PR_TRY(launch_backward(ws->views.as<ViewDev>(), n, ws->offs.as<long long>(), blk[n], nullptr,
                           shade_features(ws->h_views.p, n), st, ws->h_views.p));
    PR_TRY(cudaStreamSynchronize(st));
    return PR_OK;
}

namespace {

// The checks of one view of the display step (shared by the single and
// batched calls).
bool unfoveate_view_ok(const pr_view *view, const float *rgb, const float *out, int Wd, int Hd, int method,
                       float sigma)
{
    if (!view || !rgb || !out)
        return false;
    const pr_view &v = *view;
    if (v.W < 1 || v.H < 1 || v.W > 16384 || v.H > 16384 || Wd < 1 || Hd < 1 || Wd > 16384 || Hd > 16384)
        return false;
    if (v.mode < PR_CLASSIC || v.mode > PR_BOTH || !(v.alpha >= 1.f && v.alpha <= 5.f) ||
        !(v.fovea[0] >= 0.f && v.fovea[0] <= 1.f && v.fovea[1] >= 0.f && v.fovea[1] <= 1.f))
        return false;
    if (method != PR_UNFOVEATE_MIP_CUBIC && method != PR_UNFOVEATE_PROJECTED)
        return false;
    if (method == PR_UNFOVEATE_PROJECTED && !(sigma > 0.f && std::isfinite(sigma)))
        return false;
    return is_device_ptr(rgb) && is_device_ptr(out);
}

}  // namespace

pr_status pr_unfoveate(pr_workspace *ws, const pr_view *view, const float *rgb, float *out,
                       const pr_unfoveate_params *params, void *stream)
{
    if (!ws || !params)
        return PR_ERR_INVALID_ARG;
    const pr_unfoveate_params &p = *params;
    if (!unfoveate_view_ok(view, rgb, out, p.Wd, p.Hd, p.method, p.sigma))
        return PR_ERR_INVALID_ARG;
    const pr_view &v = *view;
    cudaStream_t st = (cudaStream_t)stream;
    // scratch: the MIP pyramid, or the projected filter's table of q (2 floats per pixel)
    PR_TRY(ensure(ws->mip, sizeof(float) * mip_pyramid_floats(v.W, v.H)));
    float *pyr = ws->mip.as<float>();
    PR_TRY(launch_unfoveate(p.method, v.W, v.H, v.mode, v.fovea[0], v.fovea[1], v.alpha,
                            v.foveation ? v.foveation->lut : nullptr, v.foveation ? v.foveation->n : 0, p.Wd, p.Hd,
                            p.sigma, rgb, pyr, out, st));
    return PR_OK;
}

pr_status pr_unfoveate_batch(pr_workspace *ws, const pr_unfoveate_entry *entries, int32_t n,
                             const pr_unfoveate_params *params, void *stream)
{
    if (!ws || !params || n < 0 || (n > 0 && !entries))
        return PR_ERR_INVALID_ARG;
    const pr_unfoveate_params &p = *params;
    std::vector<DisplayEntry> e((size_t)n);
    for (int k = 0; k < n; ++k) {
        const pr_unfoveate_entry &x = entries[k];
        if (!unfoveate_view_ok(x.view, x.rgb, x.out, x.Wd, x.Hd, p.method, p.sigma))
            return PR_ERR_INVALID_ARG;
        const pr_view &v = *x.view;
        DisplayEntry &d = e[(size_t)k];
        d.W = v.W;
        d.H = v.H;
        d.mode = v.mode;
        d.fx = v.fovea[0];
        d.fy = v.fovea[1];
        d.alpha = v.alpha;
        d.p_lut = v.foveation ? v.foveation->lut : nullptr;
        d.p_n = v.foveation ? v.foveation->n : 0;
        d.Wd = x.Wd;
        d.Hd = x.Hd;
        d.rgb = x.rgb;
        d.out = x.out;
    }
    if (n == 0)
        return PR_OK;
    cudaStream_t st = (cudaStream_t)stream;
    // the previous batch call's table copy must be done before its pinned
    // source is rewritten (or freed by a regrowth)
    if (ws->disp_ev_pending) {
        PR_TRY(cudaEventSynchronize(ws->disp_ev));
        ws->disp_ev_pending = false;
    }
    const size_t tb = display_batch_table_bytes(n);
    PR_TRY(ws->h_disp.ensure(tb));
    PR_TRY(ensure(ws->disp, tb));
    PR_TRY(ensure(ws->mip, sizeof(float) * std::max<size_t>(display_batch_scratch_floats(p.method, e.data(), n), 1)));
    if (!ws->disp_ev)
        PR_TRY(cudaEventCreateWithFlags(&ws->disp_ev, cudaEventDisableTiming));
    PR_TRY(launch_unfoveate_batch(p.method, p.sigma, e.data(), n, ws->mip.as<float>(), ws->h_disp.p, ws->disp.p,
                                  st));
    if (p.method == PR_UNFOVEATE_MIP_CUBIC) {  // the only form that copies the table
        PR_TRY(cudaEventRecord(ws->disp_ev, st));
        ws->disp_ev_pending = true;
    }
    return PR_OK;
}

pr_status pr_workspace_create(pr_workspace **out)
{
    if (!out)
        return PR_ERR_INVALID_ARG;
    *out = new (std::nothrow) pr_workspace;
    return *out ? PR_OK : PR_ERR_OOM;
}

void pr_workspace_free(pr_workspace *ws)
{
    if (ws) {
        cudaDeviceSynchronize();
        delete ws;
    }
}

pr_status pr_rasterize_batch(pr_workspace *ws, const pr_batch_view *views, int32_t n, const pr_params *params,
                             void *stream)
{
    if (!ws)
        return PR_ERR_INVALID_ARG;
    return run_batch(ws, views, n, params, true, (cudaStream_t)stream);
}

pr_status pr_frame_batch(pr_workspace *ws, const pr_batch_view *views, int32_t n, const pr_params *params,
                         const pr_frame_grad *grads, void *stream)
{
    if (!ws)
        return PR_ERR_INVALID_ARG;
    return run_batch(ws, views, n, params, true, (cudaStream_t)stream, grads);
}

pr_status pr_graph_capture_frame(pr_workspace *ws, const pr_batch_view *views, int32_t n, const pr_params *params,
                                 const pr_frame_grad *grads, void *stream, pr_graph **out)
{
    if (!ws || !out)
        return PR_ERR_INVALID_ARG;
    *out = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    if (!st)
        return PR_ERR_INVALID_ARG;  // the legacy default stream cannot be captured
    // eager run: sizes every buffer and warms up the kernels
    pr_status s = run_batch(ws, views, n, params, true, st, grads);
    if (s != PR_OK)
        return s;
    pr_params prm = default_params(params);
    BatchPlan P;
    s = plan_batch(views, n, prm, P, grads);
    if (s != PR_OK)
        return s;
    for (const auto &o : P.out)
        if (o.id_host || o.depth_host || o.rgb_host)
            return PR_ERR_INVALID_ARG;  // graphs need device outputs
    pr_graph *g = new (std::nothrow) pr_graph;
    if (!g)
        return PR_ERR_OOM;
    g->ws = ws;
    g->npix = P.npix;
    g->buffers = ws->buffer_set();
    // the graph's own copy of the view and offset tables, written once here:
    // replays upload nothing, and later calls on the workspace cannot change it
    const int nv = (int)P.vd.size();
    fill_tables(ws, P, true);
    cudaError_t e = ensure(g->views, sizeof(ViewDev) * nv);
    if (e == cudaSuccess)
        e = ensure(g->offs, sizeof(long long) * 4 * (nv + 1));
    if (e == cudaSuccess)
        e = g->h_cnt.ensure(1);
    if (e == cudaSuccess)
        std::memcpy(g->h_cnt.p, ws->h_cnt.p, sizeof(Counters));  // the eager run's, until the first replay
    if (e == cudaSuccess)
        e = cudaMemcpy(g->views.p, ws->h_views.p, sizeof(ViewDev) * nv, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(g->offs.p, ws->h_offs.p, sizeof(long long) * 4 * (nv + 1), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        delete g;
        cudaGetLastError();
        return from_cuda(e);
    }
    e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        delete g;
        cudaGetLastError();
        return from_cuda(e);
    }
    g->stage_times = prm.graph_stage_times != 0;
    // a capture runs nothing: the keys keep the state the eager run left
    const long long clean_n = ws->keys_clean_n;
    s = enqueue_batch(ws, P, prm.seg, true, st, g->views.as<ViewDev>(), g->offs.as<long long>(), g->stage_times,
                      g->h_cnt.p);
    ws->keys_clean_n = clean_n;
    g->reader_resets = keys_reset_by_reader(P.npix);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(st, &graph);
    if (s != PR_OK || e != cudaSuccess) {
        if (graph)
            cudaGraphDestroy(graph);
        delete g;
        cudaGetLastError();
        return s != PR_OK ? s : from_cuda(e);
    }
    g->graph = graph;
    e = cudaGraphInstantiate(&g->exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        delete g;
        cudaGetLastError();
        return from_cuda(e);
    }
    *out = g;
    return PR_OK;
}

pr_status pr_graph_capture_batch(pr_workspace *ws, const pr_batch_view *views, int32_t n, const pr_params *params,
                                 void *stream, pr_graph **out)
{
    return pr_graph_capture_frame(ws, views, n, params, nullptr, stream, out);
}

pr_status pr_graph_enqueue(pr_graph *g, void *stream)
{
    if (!g)
        return PR_ERR_INVALID_ARG;
    pr_workspace *ws = g->ws;
    if (ws->buffer_set() != g->buffers)
        return PR_ERR_INVALID_ARG;  // a later call regrew the workspace: the graph's pointers are stale
    // a graph whose reader sets the keys back clears none at its start: if
    // the work before it (a frame whose keys fit in L2, an interrupted
    // sequence) left keys in use, they are cleared here first
    if (g->reader_resets && ws->keys_clean_n < g->npix)
        PR_TRY(cudaMemsetAsync(ws->keys.p, 0xFF, sizeof(unsigned long long) * (size_t)g->npix,
                               (cudaStream_t)stream));
    PR_TRY(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
    ws->keys_clean_n = g->reader_resets ? std::max(ws->keys_clean_n, g->npix) : 0;
    return PR_OK;
}

pr_status pr_graph_launch(pr_graph *g, void *stream)
{
    pr_status s = pr_graph_enqueue(g, stream);
    if (s != PR_OK)
        return s;
    PR_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    return pr_graph_status(g);
}

pr_status pr_graph_status(pr_graph *g)
{
    if (!g)
        return PR_ERR_INVALID_ARG;
    pr_workspace *ws = g->ws;
    const Counters &c = *g->h_cnt.p;
    ws->stats.tests = c.tests;
    ws->stats.hits = c.hits;
    ws->stats.pairs = c.pairs_total;
    ws->stats.items = c.items_total;
    ws->stats.culled = c.culled;
    ws->stats.flagged = c.flagged;
    ws->stats.changed = c.changed;
    {
        unsigned b = c.depth_err_bits;
        float e;
        std::memcpy(&e, &b, sizeof e);
        ws->stats.fp64_depth_err = e;
    }
    ws->stats.pixels = (uint64_t)g->npix;
    if (g->stage_times) {
        ws->read_stage_times();
    } else {
        for (int k = 0; k < 8; ++k)
            ws->stats.stage_ms[k] = 0.f;
    }
    if (c.status & ST_TIMEOUT)
        return PR_ERR_TIMEOUT;
    if (c.status & ST_NONFINITE)
        return PR_ERR_NONFINITE;  // a scene updated with a non-finite value: its triangles were culled
    if (c.status & (ST_OVERFLOW_PAIRS | ST_OVERFLOW_ITEMS | ST_OVERFLOW_FLAGS))
        return PR_ERR_OVERFLOW;
    return PR_OK;
}

void pr_graph_free(pr_graph *g)
{
    if (g) {
        cudaDeviceSynchronize();  // a replay in flight still writes the graph's status copy
        if (g->exec)
            cudaGraphExecDestroy(g->exec);
        if (g->graph)
            cudaGraphDestroy(g->graph);
        delete g;
    }
}

pr_status pr_scene_stats(const pr_scene *sc, pr_stats *out)
{
    if (!sc || !out)
        return PR_ERR_INVALID_ARG;
    *out = sc->ws.stats;
    return PR_OK;
}

pr_status pr_workspace_stats(const pr_workspace *ws, pr_stats *out)
{
    if (!ws || !out)
        return PR_ERR_INVALID_ARG;
    *out = ws->stats;
    return PR_OK;
}

pr_status pr_debug_bounds(const pr_scene *sc, int32_t *pix_box, float *t_range)
{
    if (!sc || !pix_box || !t_range)
        return PR_ERR_INVALID_ARG;
    const pr_workspace &ws = sc->ws;
    const long long T = ws.last_T;
    if (T != sc->T || !ws.tbox.p)
        return PR_ERR_INVALID_ARG;
    std::vector<int4> tb(T);
    std::vector<float4> rec(T * kRecF4);
    PR_TRY(cudaDeviceSynchronize());
    PR_TRY(cudaMemcpy(tb.data(), ws.tbox.p, sizeof(int4) * T, cudaMemcpyDeviceToHost));
    PR_TRY(cudaMemcpy(rec.data(), ws.rec.p, sizeof(float4) * kRecF4 * T, cudaMemcpyDeviceToHost));
    for (long long k = 0; k < T; ++k) {
        const int4 b = tb[k];
        pix_box[4 * k + 0] = b.x & 0xffff;
        pix_box[4 * k + 1] = b.y & 0xffff;
        pix_box[4 * k + 2] = (b.x >> 16) & 0xffff;
        pix_box[4 * k + 3] = (b.y >> 16) & 0xffff;  // a culled triangle has the empty box [1, 0]
        t_range[2 * k + 0] = rec[k * kRecF4 + 5].x;
        t_range[2 * k + 1] = rec[k * kRecF4 + 5].y;
    }
    return PR_OK;
}

pr_status pr_debug_halfplanes(const pr_scene *sc, float *hp_out, int32_t *info)
{
    if (!sc || !hp_out || !info)
        return PR_ERR_INVALID_ARG;
    const pr_workspace &ws = sc->ws;
    const long long T = ws.last_T;
    if (T != sc->T || !ws.tbox.p || !ws.hp.p)
        return PR_ERR_INVALID_ARG;
    std::vector<int4> tb(T);
    PR_TRY(cudaDeviceSynchronize());
    PR_TRY(cudaMemcpy(tb.data(), ws.tbox.p, sizeof(int4) * T, cudaMemcpyDeviceToHost));
    PR_TRY(cudaMemcpy(hp_out, ws.hp.p, sizeof(float4) * kMaxHp * T, cudaMemcpyDeviceToHost));
    for (long long k = 0; k < T; ++k)
        info[k] = tb[k].z & 0x1ff;
    return PR_OK;
}

int32_t pr_debug_catch_interval(const pr_view *view, const float *S, const float *E, float *t_out)
{
    if (!view || !S || !E || !t_out)
        return -1;
    float3 s3[3], d3[3];
    for (int k = 0; k < 3; ++k) {
        s3[k] = make_float3(S[3 * k], S[3 * k + 1], S[3 * k + 2]);
        d3[k] = make_float3(E[3 * k] - S[3 * k], E[3 * k + 1] - S[3 * k + 1], E[3 * k + 2] - S[3 * k + 2]);
    }
    const float t_hi = std::min(1.f, view->d[0] + view->d[1]);
    float lo = 0.f, hi = 0.f;
    const bool ok = catch_interval(s3, d3, view->tan_x, view->tan_y, view->d[0], view->d[1], 0.f, t_hi, lo, hi);
    t_out[0] = lo;
    t_out[1] = hi;
    return ok ? 1 : 0;
}

}  // extern "C"
