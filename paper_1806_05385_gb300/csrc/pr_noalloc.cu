// pr_noalloc.cu -- pr_rasterize_noalloc: stages (a)-(c) of one view with all
// scratch in a fixed, file-scope device array instead of allocated buffers.
//
// Who needs it: a caller that may not allocate device memory -- a real-time
// frame loop (VR compositor, game engine) in which cudaMalloc/cudaFree would
// synchronise the device and stall the frame, or a host that owns all GPU
// memory up front and hands libraries none.  Such a caller still passes its
// own device input arrays and output buffers; everything else lives in
// g_noalloc_scratch.
//
// The array is kNoAllocBytes (64 MiB) and is held by every GPU that loads
// the library until the process exits.  Every call on a device shares it and
// it keeps the last call's contents, so each call clears what must start at
// zero, and calls whose work overlaps on the GPU (other streams, or another
// host thread) race on it: serialise them.  The host-side name of the array
// is only a stand-in for the device symbol, so its device address is looked
// up with cudaGetSymbolAddress once per device, on the first call made on
// that device (with that device current).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "pr_launch.h"

using namespace pr;

namespace {

constexpr size_t kNoAllocBytes = 64ull << 20;
constexpr int kMaxDevices = 64;

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {

void *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of g_noalloc_scratch on the current device (set up once).
cudaError_t scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= kMaxDevices)
        return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess)
            return e;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

bool on_device(const void *p)
{
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

pr_status status_of(cudaError_t e)
{
    if (e == cudaSuccess)
        return PR_OK;
    cudaGetLastError();
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver)
        return PR_ERR_NO_CUDA;
    return PR_ERR_CUDA;
}

#define NA_TRY(expr)                          \
    do {                                      \
        cudaError_t _e = (expr);              \
        if (_e != cudaSuccess)                \
            return status_of(_e);             \
    } while (0)

// Carves aligned regions out of the arena; fails once it is exhausted.
struct Carver {
    size_t off = 0;
    bool ok = true;
    size_t take(size_t bytes)
    {
        const size_t at = (off + 255) & ~(size_t)255;
        if (at + bytes > kNoAllocBytes) {
            ok = false;
            return 0;
        }
        off = at + bytes;
        return at;
    }
};

// View constants of pr_view from the shared validation of every entry
// point, with the scene arrays in the arena.
pr_status view_constants(const pr_view &in, int tile, int bound, const float4 *vtx, const float4 *col4,
                         const int4 *tri4, long long V, long long T, ViewDev &v)
{
    const pr_status s = derive_view(in, tile, bound, 0, v);
    if (s != PR_OK)
        return s;
    v.T = (int)T;
    v.V = (int)V;
    v.vtx = vtx;
    v.col4 = col4;
    v.tri4 = tri4;
    return PR_OK;
}

}  // namespace

extern "C" pr_status pr_rasterize_noalloc(const float *pos, const float *vel, const float *col, const int32_t *tri,
                                          int64_t V, int64_t T, const pr_view *view, const pr_params *params,
                                          uint32_t *id_out, float *depth_out, void *stream)
{
    if (!view || V < 1 || T < 0 || V > (1ll << 30) || T > (1ll << 30))
        return PR_ERR_INVALID_ARG;
    if (!on_device(pos) || !on_device(vel) || !on_device(col) || (T > 0 && !on_device(tri)) ||
        (id_out && !on_device(id_out)) || (depth_out && !on_device(depth_out)))
        return PR_ERR_INVALID_ARG;  // device buffers only: staging host memory would need allocations
    if (params && params->fp64_retest != 0)
        return PR_ERR_INVALID_ARG;  // the FP64 re-test's flag buffers are not carved from the arena
    cudaStream_t st = (cudaStream_t)stream;
    const int tile = params && params->tile ? params->tile : 16;
    const int bound = params ? params->bound : PR_BOUND_ZENON;
    const int seg = std::min(params && params->seg > 0 ? params->seg : 256, kMaxSeg);

    void *base = nullptr;
    NA_TRY(scratch_address(&base));
    char *arena = static_cast<char *>(base);

    // layout of this call in the arena
    const long long W = view->W, H = view->H;
    if (W < 1 || H < 1 || W > 16384 || H > 16384 || (tile != 8 && tile != 16 && tile != 32))
        return PR_ERR_INVALID_ARG;
    const long long nt = ((W + tile - 1) / tile) * ((H + tile - 1) / tile), np = W * H, Tn = std::max<int64_t>(T, 1);
    Carver c;
    const size_t o_views = c.take(sizeof(ViewDev)), o_offs = c.take(sizeof(long long) * 8);
    const size_t o_cnt = c.take(sizeof(Counters)), o_heads = c.take(sizeof(int) * 8);
    const size_t o_vtx = c.take(sizeof(float4) * 2 * V), o_col = c.take(sizeof(float4) * V);
    const size_t o_idx = c.take(sizeof(int4) * Tn);
    const size_t o_rec = c.take(sizeof(float4) * kRecF4 * Tn), o_hp = c.take(sizeof(float4) * kMaxHp * Tn);
    const size_t o_tbox = c.take(sizeof(int4) * Tn), o_cand = c.take(8 * Tn), o_cand_off = c.take(8 * (Tn + 1));
    const size_t o_binned = c.take(sizeof(int) * Tn);
    const size_t o_tile_box = c.take(sizeof(float4) * nt), o_tile_cnt = c.take(8 * nt);
    const size_t o_scan = c.take(8 * (nt + 1)), o_fill = c.take(4 * nt);
    const size_t o_sums = c.take(8 * (scan_block_sums_needed(Tn) + scan_block_sums_needed(nt)));
    const size_t o_keys = c.take(8 * np);
    if (!c.ok)
        return PR_ERR_INVALID_ARG;  // the frame's fixed scratch exceeds the 64 MiB arena
    // the rest: work items and bin entries
    const long long rest = (long long)kNoAllocBytes - (long long)((c.off + 255) & ~(size_t)255) - 512;
    const long long item_fixed = nt + 1024;
    if (rest < (long long)(16 * item_fixed + 21 * (2 * Tn + nt)))
        return PR_ERR_OVERFLOW;  // too little room left for the bins of this frame
    // per bin entry: the entry (8 B) and its listed hit (8 B entry + 4 B tile)
    const long long cap_pairs = (rest - 16 * item_fixed) / (20 + 16 / seg + 1);
    const long long cap_items = item_fixed + cap_pairs / seg + 1;
    const size_t o_items = c.take(sizeof(int4) * cap_items), o_tris = c.take(8 * cap_pairs);
    const size_t o_hit_e = c.take(8 * cap_pairs), o_hit_t = c.take(4 * cap_pairs);
    if (!c.ok)
        return PR_ERR_OVERFLOW;  // the bins' alignment padding did not fit either

    float4 *vtx = (float4 *)(arena + o_vtx), *col4 = (float4 *)(arena + o_col);
    int4 *tri4 = (int4 *)(arena + o_idx);
    ViewDev v;
    pr_status s = view_constants(*view, tile, bound, vtx, col4, tri4, V, T, v);
    if (s != PR_OK)
        return s;
    const int fov_bound = params ? params->fov_bound : PR_FOV_SECTOR;
    if (fov_bound < PR_FOV_SECTOR || fov_bound > PR_FOV_RECURSIVE)
        return PR_ERR_INVALID_ARG;
    v.fov_bound = fov_bound;
    v.id_out = id_out;
    v.depth_out = depth_out;
    long long offs[8] = {0, T, 0, nt, 0, np, 0, 0};  // tri, tile, pixel offsets of the one view

    ViewDev *dv = (ViewDev *)(arena + o_views);
    long long *doffs = (long long *)(arena + o_offs);
    Counters *cnt = (Counters *)(arena + o_cnt);
    v.scene_status = &cnt->status;  // stage (a) culls every triangle if the scene check below finds a non-finite value
    int *heads = (int *)(arena + o_heads);
    unsigned long long *cand = (unsigned long long *)(arena + o_cand), *cand_off = (unsigned long long *)(arena + o_cand_off);
    unsigned long long *tile_cnt = (unsigned long long *)(arena + o_tile_cnt), *scan = (unsigned long long *)(arena + o_scan);
    float4 *rec = (float4 *)(arena + o_rec), *hp = (float4 *)(arena + o_hp), *tile_box = (float4 *)(arena + o_tile_box);
    int4 *tbox = (int4 *)(arena + o_tbox), *items = (int4 *)(arena + o_items);
    unsigned *fill = (unsigned *)(arena + o_fill);
    unsigned long long *pairs = (unsigned long long *)(arena + o_tris);
    unsigned long long *hit_entry = (unsigned long long *)(arena + o_hit_e);
    unsigned *hit_tile = (unsigned *)(arena + o_hit_t);
    unsigned long long *keys = (unsigned long long *)(arena + o_keys);
    // look-back states of the two scans: candidate tiles, then tile counts
    unsigned long long *state_a = (unsigned long long *)(arena + o_sums), *state_b = state_a + scan_block_sums_needed(Tn);

    // host-side constants go up by plain (pageable) copies; they complete
    // before the call returns, so the stack buffers may go out of scope
    NA_TRY(cudaMemcpyAsync(dv, &v, sizeof v, cudaMemcpyHostToDevice, st));
    NA_TRY(cudaMemcpyAsync(doffs, offs, sizeof offs, cudaMemcpyHostToDevice, st));
    const long long *tri_offs = doffs, *tile_offs = doffs + 2, *pix_offs = doffs + 4;
    // what must start at zero, the keys at ~0 (the arena keeps the previous
    // call's contents), and the tiles' display boxes
    NA_TRY(launch_frame_init(dv, 1, tile_offs, tile_box, cnt, heads, tile_cnt, fill, nt, state_a, scan_state_words(T),
                             state_b, scan_state_words(nt), nullptr, 0, keys, np, nullptr, 0, st));
    NA_TRY(launch_scene_pack(pos, vel, col, V, vtx, col4, st));
    NA_TRY(launch_scene_idx(tri, T, V, tri4, cnt, st));
    NA_TRY(launch_scene_check(vtx, col4, V, &cnt->status, st));
    int *binned = (int *)(arena + o_binned);
    NA_TRY(launch_bound(dv, 1, tri_offs, T, rec, hp, tbox, cand, binned, cnt, st));
    if (fov_bound != PR_FOV_SECTOR && (view->mode == PR_FOVEATED || view->mode == PR_BOTH))
        NA_TRY(launch_paper_fov(dv, 1, tri_offs, T, rec, hp, tbox, cand, st));
    NA_TRY(launch_scan(cand, cand_off, state_a, T, 0, cnt, st, true, binned, &cnt->binned));
    NA_TRY(launch_bin_count(dv, 1, tri_offs, T, binned, cand_off, rec, hp, tbox, tile_box, tile_cnt, hit_entry,
                            hit_tile, cap_pairs, cnt, st));
    ItemsOut io;  // the scan of the tile counts also emits the work items
    io.views = dv;
    io.nviews = 1;
    io.tile_offs = tile_offs;
    io.items = items;
    io.cap_items = cap_items;
    io.cap_pairs = cap_pairs;
    NA_TRY(launch_scan(tile_cnt, scan, state_b, nt, seg, cnt, st, true, nullptr, nullptr, &io));
    NA_TRY(launch_bin_scatter(hit_entry, hit_tile, scan, fill, pairs, cap_pairs, nt, cnt, st));
    NA_TRY(launch_sort_items(items, scan, nt, cap_items, seg, pairs, cnt, st));
    NA_TRY(launch_fragment(tile, false, dv, items, scan, 0, nt, cap_items, heads, pairs, rec, keys, nullptr,
                           nullptr, cnt, fragment_grid(tile, false), st));
    NA_TRY(launch_resolve(dv, 1, pix_offs, np, keys, false, st));
    Counters h;
    NA_TRY(cudaMemcpyAsync(&h, cnt, sizeof h, cudaMemcpyDeviceToHost, st));
    NA_TRY(cudaStreamSynchronize(st));
    if (h.status & ST_TIMEOUT)
        return PR_ERR_TIMEOUT;  // a scan's bounded wait ran out: its offsets and the bins behind them are invalid
    if (h.status & ST_NONFINITE)
        return PR_ERR_NONFINITE;
    if (h.status & ST_BAD_INDEX)
        return PR_ERR_INVALID_ARG;
    if (h.status & (ST_OVERFLOW_PAIRS | ST_OVERFLOW_ITEMS))
        return PR_ERR_OVERFLOW;  // the bins of this frame do not fit the fixed arena
    return PR_OK;
}
