// pr_launch.h -- host-side launchers of the libpr kernels (one per stage).
#pragma once

#include <cuda_runtime.h>

#include "pr_internal.cuh"

namespace pr {

// scene upload: [V][3] arrays -> 32-byte vertex records (vtx, 2 float4 per
// vertex) and float4 colours, [T][3] indices -> int4; finiteness and index
// checks.  launch_scene_set replaces one array (which: 0 pos, 1 vel, 2 col).
cudaError_t launch_scene_pack(const float *pos, const float *vel, const float *col, long long V, float4 *vtx,
                              float4 *col4, cudaStream_t st);
cudaError_t launch_scene_idx(const int *tri, long long T, long long V, int4 *tri4, Counters *cnt, cudaStream_t st);
cudaError_t launch_scene_set(const float *src, int which, long long V, float4 *vtx, float4 *col4, cudaStream_t st);
cudaError_t launch_scene_check(const float4 *vtx, const float4 *col4, long long V, unsigned *status, cudaStream_t st);
// one scene of a batched update: its records, status word and new arrays (null: keep)
struct SceneUpdate {
    float4 *vtx, *col4;
    unsigned *status;
    const float *pos, *vel, *col;
    long long V;
};
constexpr int kSceneUpdateChunk = 64;  // scenes per launch (passed by value)
cudaError_t launch_scene_update_batch(const SceneUpdate *u, int n, cudaStream_t st);

// stage (a): per-triangle bounds (the tiles' display boxes come with the frame init)
// binned: the triangles with candidate tiles are appended here (cnt->binned)
cudaError_t launch_bound(const ViewDev *views, int nviews, const long long *tri_offs, long long ttot, float4 *rec,
                         float4 *hp, int4 *tbox, unsigned long long *cand, int *binned, Counters *cnt,
                         cudaStream_t st);
// the paper's foveation edge bounds for the views that select them (after launch_bound)
cudaError_t launch_paper_fov(const ViewDev *views, int nviews, const long long *tri_offs, long long ttot,
                             const float4 *rec, float4 *hp, int4 *tbox, unsigned long long *cand, cudaStream_t st);

// stage (b): tile binning -- count pass (tile counts, and every hit appended to the hit list)
// over the binned triangles (cand_off: prefix of their candidate counts), then after the scan
// the scatter of the list into the bins
cudaError_t launch_bin_count(const ViewDev *views, int nviews, const long long *tri_offs, long long ttot,
                             const int *binned, const unsigned long long *cand_off, const float4 *rec,
                             const float4 *hp, const int4 *tbox, const float4 *tile_box, unsigned long long *tile_cnt,
                             unsigned long long *hit_entry, unsigned *hit_tile, long long cap_pairs, Counters *cnt,
                             cudaStream_t st);
cudaError_t launch_bin_scatter(const unsigned long long *hit_entry, const unsigned *hit_tile,
                               const unsigned long long *scan, unsigned int *fill, unsigned long long *pairs,
                               long long cap_pairs, long long ntiles, Counters *cnt, cudaStream_t st);
// Where the scan of the tile counts writes the fragment stage's work items.
struct ItemsOut {
    const ViewDev *views = nullptr;
    int nviews = 0;
    const long long *tile_offs = nullptr;
    int4 *items = nullptr;
    long long cap_items = 0, cap_pairs = 0;
};
// state_zeroed: the caller cleared the ticket and flags (state[0, 1 + nb)).
// gather: scan in[gather[i]]; n_dev: the count is min(*n_dev, n) (device).
// items (with seg > 0): also emit each tile's work items and the totals.
cudaError_t launch_scan(const unsigned long long *in, unsigned long long *out, unsigned long long *state, long long n,
                        int seg, Counters *cnt, cudaStream_t st, bool state_zeroed = false,
                        const int *gather = nullptr, const unsigned long long *n_dev = nullptr,
                        const ItemsOut *items = nullptr);
// the start of a frame: clears, the first npix keys to ~0 (0: none, where the
// last frames' readers left them so), tile display boxes (one launch)
cudaError_t launch_frame_init(const ViewDev *views, int nviews, const long long *tile_offs, float4 *tile_box,
                              Counters *cnt, int *heads, unsigned long long *tile_cnt, unsigned *fill, long long ntiles,
                              unsigned long long *state_a, long long nstate_a, unsigned long long *state_b,
                              long long nstate_b, unsigned *flag_bits, long long nflag, unsigned long long *keys,
                              long long npix, float *loss_part, long long nloss, cudaStream_t st);
size_t scan_block_sums_needed(long long n);
// a scan whose look-back waits on a tile that never runs (status word out)
cudaError_t scan_timeout_probe(cudaStream_t st, unsigned *status);
// words of a scan's state that must start at zero (ticket and flags)
long long scan_state_words(long long n);
// sorts every item's run of bin entries (nearest first); runs <= kMaxSeg
cudaError_t launch_sort_items(const int4 *items, const unsigned long long *scan, long long ntiles, long long cap_items,
                              int seg, unsigned long long *pairs, const Counters *cnt, cudaStream_t st);

// stage (c): per-fragment ray casting, FP64 re-test, resolve
cudaError_t launch_fragment(int S, bool flag, const ViewDev *views, const int4 *items, const unsigned long long *scan,
                            long long tile_lo, long long tile_hi, long long cap_items, int *head,
                            const unsigned long long *pairs, const float4 *rec, unsigned long long *keys,
                            unsigned *flag_bits, long long *flag_list, Counters *cnt, int grid, cudaStream_t st);
int fragment_grid(int S, bool flag);
cudaError_t launch_retest(const ViewDev *views, int nviews, const long long *pix_offs, const unsigned long long *scan,
                          const unsigned long long *tile_cnt, const unsigned long long *pairs, const float4 *rec,
                          const long long *flag_list, unsigned long long *keys, long long cap_pairs, Counters *cnt,
                          cudaStream_t st);
// id and depth of every pixel from its key (reset_keys: the key set back to ~0)
cudaError_t launch_resolve(const ViewDev *views, int nviews, const long long *pix_offs, long long npix,
                           unsigned long long *keys, bool reset_keys, cudaStream_t st);

// stages (d) and (e)
// keys: resolve them too (reset_keys: each set back to ~0), or null: read id_in; adjoint: a training frame,
// run stage (e) for the views with a gradient from the same pixel hit
// feat: shade_features of the launch's views (which optional paths to build in)
int shade_features(const ViewDev *vd, int n);
// host_views: the host copy of the device table `views` (same contents), or
// null; with one, a launch of up to kParamViews views passes them as a
// kernel parameter
cudaError_t launch_shade(const ViewDev *views, int nviews, const long long *blk_offs, long long nblocks,
                         unsigned long long *keys, bool reset_keys, bool adjoint, const Counters *frame_cnt, int feat,
                         cudaStream_t st, const ViewDev *host_views = nullptr);
// a training frame's losses: each view's partial sums (loss_part) added into
// its loss, once (skipped when the frame's forward overflowed)
cudaError_t launch_loss_finalize(const ViewDev *views, int nviews, const Counters *frame_cnt, cudaStream_t st);
// frame_cnt: the counters of the frame whose forward ran just before in the
// same sequence (the adjoint is skipped if it overflowed), or null.
cudaError_t launch_backward(const ViewDev *views, int nviews, const long long *blk_offs, long long nblocks,
                            const Counters *frame_cnt, int feat, cudaStream_t st, const ViewDev *host_views = nullptr);

// display step: unfoveation of a framebuffer image (pyramid: scratch of
// mip_pyramid_floats(W, H) floats for the MIP method)
size_t mip_pyramid_floats(int W, int H);
cudaError_t launch_unfoveate(int method, int W, int H, int mode, float fx, float fy, float alpha, const float *p_lut,
                             int p_n, int Wd, int Hd, float sigma, const float *rgb, float *pyramid, float *out,
                             cudaStream_t st);
// the batched display step: n views, each with its own size, mode and
// display size, one method and filter width for all
struct DisplayEntry {
    int W, H, mode;
    float fx, fy, alpha;
    const float *p_lut;  // sampled p (device) or null
    int p_n;
    int Wd, Hd;
    const float *rgb;  // device [3][H][W]
    float *out;        // device [3][Hd][Wd]
};
// scratch floats of the batch (MIP: each view's pyramid, 16-byte aligned;
// the projected filter needs none)
size_t display_batch_scratch_floats(int method, const DisplayEntry *e, int n);
// bytes of the host and device tables of a batch of n views
size_t display_batch_table_bytes(int n);
// Fills the table into h_table (pinned host memory, display_batch_table_bytes(n)
// bytes; the caller makes sure a previous copy out of it has finished), copies
// it to d_table on st and launches the batch.
cudaError_t launch_unfoveate_batch(int method, float sigma, const DisplayEntry *e, int n, float *scratch,
                                   void *h_table, void *d_table, cudaStream_t st);
// measured FP32 FMA throughput of the current device, TFLOP/s
cudaError_t measure_fma_peak(cudaStream_t st, double *tflops);

// device samples of a foveation handle (defined with the handle)
const float *pr_foveation_samples(const pr_foveation *f, int *n);

// validation of a view and its device constants (all but the scene's
// arrays and sizes, which the caller sets); PR_ERR_INVALID_ARG for any
// out-of-range field, tile or bound kind
pr_status derive_view(const pr_view &in, int tile, int bound, int fp64, ViewDev &v);

}  // namespace pr
