/*
 * pr.h -- C ABI of the GB300 perceptual-rasterization library (libpr.so).
 *
 * Perceptual rasterization (Ritschel, Friston, Steed 2018) draws a frame in
 * which every pixel has its own time (rolling display, Sec. 3.1.2) and its
 * own ray through a continuously foveated image (Sec. 3.1.1), by casting
 * that pixel's ray against each triangle moved to that time (Sec. 3.2,
 * "Intersection"), but only for the pixels inside a tight space-time-fovea
 * bound of the triangle (Sec. 4).  This library runs that hot path on one
 * GPU in five stages: (a) per-triangle bounds, (b) tile binning, (c) the
 * per-fragment ray test with a 64-bit atomicMin on depth|id, (d) deferred
 * shading and (e) its adjoint.
 *
 * Conventions shared by every entry point:
 *  - camera space: x right, y down, z forward; a pose is a row-major 4x4
 *    rigid world->camera transform [R | T]; pose0 holds at t = 0 and pose1
 *    at t = 1 of the frame interval (the start/end model-view matrices of
 *    Sec. 3.2, "Bounding").
 *  - a vertex moves linearly: world position p + t v over the frame; its
 *    camera-space position is c(t) = (1-t)(R0 p + T0) + t(R1 (p+v) + T1),
 *    the interpolation of M_s v_s and M_e v_e (Sec. 3.2).
 *  - pixel (i, j) has the unit framebuffer location u = ((i+.5)/W, (j+.5)/H)
 *    and the display location x = q(u) when foveated (else x = u), with
 *    q(u) = x_f + (u - x_f)/|u - x_f| * p(|u - x_f|), p(d) = D (d/D)^alpha,
 *    D = sqrt(2) (Sec. 3.1.1; power foveation of Sec. 5.1).
 *  - its time is t = r(x) = x . d when rolling, else 0 (Sec. 3.1.2; the joint
 *    mode takes the time at the display location, Sec. 3.1.3 / 4.3).
 *  - its camera-space ray starts at the origin with direction
 *    ((2 x0 - 1) tanX, (2 x1 - 1) tanY, 1), so the ray parameter of a hit
 *    equals its camera z, which is the stored depth (Sec. 3.2).
 *  - the nearest hit with depth > z_near wins; equal depths go to the
 *    smaller triangle id; edges are inclusive; no back-face culling.
 *
 * Memory: every pointer argument may point to device memory or to host
 * memory; the library detects which (cudaPointerGetAttributes) and stages
 * host buffers through its own device memory.  Caller-owned buffers are
 * only read or written during the call.  All work is issued on the caller's
 * stream (a cudaStream_t passed as void*, NULL = legacy default stream); a
 * call returns after its status word has been read back from the device,
 * so its outputs are complete on return.
 *
 * Errors: every entry point returns a pr_status; nothing aborts, traps or
 * throws across the ABI.  pr_status_string() names a status.
 */
#ifndef PR_H
#define PR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PR_OK = 0,
    PR_ERR_INVALID_ARG = 1, /* a size, mode, pointer or parameter is out of range */
    PR_ERR_CUDA = 2,        /* a CUDA runtime call failed (no device, launch error, ...) */
    PR_ERR_OOM = 3,         /* device allocation failed */
    PR_ERR_OVERFLOW = 4,    /* a device buffer was too small even after regrowing, or a frame
                               needs more than 2^31 - 1 bin entries (split it into smaller calls) */
    PR_ERR_TIMEOUT = 5,     /* a bounded device-side wait ran out */
    PR_ERR_NONFINITE = 6,   /* an input position/velocity/colour is NaN or Inf */
    PR_ERR_NO_CUDA = 7      /* no CUDA device is visible */
} pr_status;

typedef enum {
    PR_CLASSIC = 0,  /* t = 0, x = u: common rasterization */
    PR_ROLLING = 1,  /* t = r(u), x = u (Sec. 3.1.2) */
    PR_FOVEATED = 2, /* t = 0, x = q(u) (Sec. 3.1.1) */
    PR_BOTH = 3      /* t = r(q(u)), x = q(u) (Sec. 3.1.3) */
} pr_mode;

/* Bound of the display region a moving triangle can cover (Sec. 4.2).
 * Every kind is conservative, so the image does not depend on it (Sec. 3.2:
 * the intersection test is the same whatever bound is used); only the
 * number of ray tests does. */
typedef enum {
    PR_BOUND_ZENON = 0,    /* Sec. 4.2.4: catch-up time interval of the rolling scan, default */
    PR_BOUND_ADAPTIVE = 1, /* Sec. 4.2.3: interval of r over the projected space-time vertices */
    PR_BOUND_HULL = 2,     /* Sec. 4.2.2: convex hull of the projected space-time vertices */
    PR_BOUND_QUAD = 3,     /* Sec. 4.2.1: bounding box of the projected space-time vertices */
    PR_BOUND_TRIVIAL = 4   /* the whole viewport */
} pr_bound;

/* Foveation part of the bound (foveated and joint modes).  The triangle's
 * region is always tested in display space against each tile's display
 * image; this selects how its framebuffer extent is found and, for the
 * paper's two edge bounds, the polygon that bins tiles. */
typedef enum {
    PR_FOV_SECTOR = 0,     /* annular sector of q^-1 of the region (rigorous, default) */
    PR_FOV_SIMPLE = 1,     /* Sec. 4.1.1: each region edge displaced parallel to itself */
    PR_FOV_RECURSIVE = 2   /* Sec. 4.1.2: displaced parallel to the chord of its foveated end points */
} pr_fov_bound;

/* A foveation function given by samples (Sec. 3.1.1: p may be any
 * monotonic function, inverted numerically in a pre-processing pass; Sec. 6,
 * "Lens Distortion": p = p_c o p_l).  See pr_foveation_create. */
typedef struct pr_foveation pr_foveation;

/* One view: the camera, the two poses that bracket the frame, the fovea,
 * the display's rolling direction and the shading constants. */
typedef struct {
    int32_t W, H;         /* framebuffer size in pixels, 1..16384 */
    int32_t mode;         /* pr_mode */
    int32_t pad0;
    float tan_x, tan_y;   /* tangents of the half field of view, > 0 */
    float z_near;         /* hits need depth > z_near > 0, finite */
    float alpha;          /* foveation exponent, 1 <= alpha <= 5 (1 = identity) */
    float pose0[16];      /* world->camera at t = 0, row-major */
    float pose1[16];      /* world->camera at t = 1, row-major */
    float fovea[2];       /* x_f in unit framebuffer coordinates, in [0,1]^2 */
    float d[2];           /* rolling direction: d0, d1 >= 0 and d0 + d1 <= 1 */
    float light_w[3];     /* world-space direction towards the light (normalised by the library) */
    float k_a, k_d;       /* rgb = albedo * (k_a + k_d * max(0, n.l)) + the specular term below; finite */
    float k_s, shininess; /* rolling specular (Blinn-Phong): + k_s * max(0, n.h)^shininess on every
                             channel, h = normalize(l(t) + v), v = unit vector from the hit to the eye at
                             the pixel time (the reversed ray); k_s = 0: none; shininess >= 1 */
    const pr_foveation *foveation; /* NULL: p(d) = D (d/D)^alpha; else the sampled p of the handle
                                       (alpha is then unused) */
} pr_view;

typedef struct {
    int32_t bound;        /* pr_bound */
    int32_t tile;         /* bin tile side in pixels: 8, 16 or 32; 0 = library default (16) */
    int32_t fp64_retest;  /* 1: re-test fragments flagged by the FP32 error bound in FP64 */
    int32_t seg;          /* triangles per fragment work item; 0 = default (256), at most 1024 */
    int32_t fov_bound;    /* pr_fov_bound.  SIMPLE and RECURSIVE rest on the paper's assumption that
                             an edge's displacement is unimodal (ternary search); the library seeds
                             the search with a coarse scan and adds half a pixel, but they are not
                             rigorous for every edge (the sector bound is) */
    int32_t graph_stage_times; /* captured graphs only: 1 = keep the CUDA events between the stages as
                                  graph nodes, so every replay reports pr_stats.stage_ms; they cost
                                  tens of microseconds per replay, so by default (0) graphs carry none
                                  and a replay's stage_ms reads 0.  Eager calls always time stages. */
} pr_params;

/* Counters of the last rasterize call on a scene or workspace. */
typedef struct {
    uint64_t tests;       /* ray-triangle tests executed in stage (c) */
    uint64_t hits;        /* tests that hit (before depth resolution) */
    uint64_t pairs;       /* (triangle, tile) bin entries */
    uint64_t items;       /* fragment work items */
    uint64_t culled;      /* triangles with an empty bound */
    uint64_t flagged;     /* pixels re-tested in FP64 (precision form) */
    uint64_t changed;     /* pixels whose winner the FP64 re-test changed */
    uint64_t pixels;      /* framebuffer pixels over all views */
    float stage_ms[8];    /* device time of the last frame's stages, from CUDA events on the
                             caller's stream: [0] (a) tile boxes + bounds, [1] (b) binning
                             (count, scan, scatter, items), [2] (c) fragment kernel(s),
                             [3] FP64 re-test, [4] resolve (when not shading), [5] (d) shading
                             (which then also resolves and, in a training frame, runs the
                             (e) adjoint), [6]-[7] unused */
    float fp64_depth_err; /* precision form: largest |depth_fp32 - depth_fp64| / depth_fp64 over the
                             re-tested pixels whose winner FP64 confirmed (the FP32 error that the
                             re-test removed); 0 without the re-test */
    float pad_stats;
} pr_stats;

/* p_samples: HOST float [n + 1], p at d_k = k D / n (D = sqrt(2), the
 * largest framebuffer distance from the fovea), p_samples[0] = 0, strictly
 * increasing, finite; 2 <= n <= 65536.  The library copies them to the
 * device.  Every stage evaluates p linearly between the samples (the last
 * segment continued beyond D) and p^-1 as the exact inverse of that
 * interpolation (a binary search for the segment).  The handle must outlive
 * every call and captured graph whose views use it.  PR_ERR_INVALID_ARG for
 * samples that break the rules. */
pr_status pr_foveation_create(const float *p_samples, int32_t n, pr_foveation **out);
void pr_foveation_free(pr_foveation *f);

typedef struct pr_scene pr_scene;         /* library-owned device copy of a mesh + its scratch */
typedef struct pr_workspace pr_workspace; /* scratch of the batched entry points */

/* Copies a mesh into library-owned device memory (structure of arrays).
 * pos, vel, col: float32 [V][3] (world position at t = 0, world
 * displacement over the frame, RGB albedo); tri: int32 [T][3] vertex
 * indices in [0, V).  V >= 1 and T >= 0 up to 2^30.  The caller keeps
 * ownership of its arrays.  Returns PR_ERR_NONFINITE if a position,
 * velocity or colour is not finite, PR_ERR_INVALID_ARG for an index out of
 * range.  The mesh is the world-space input of Sec. 3.2 ("Bounding").  */
pr_status pr_scene_upload(const float *pos, const float *vel, const float *col, const int32_t *tri,
                          int64_t V, int64_t T, void *stream, pr_scene **out);

/* Replaces the positions, velocities and colours of an uploaded scene
 * (same V); any pointer may be NULL to keep that array.  Used to step the
 * scene in optimisation loops without re-uploading the indices.  Arrays
 * may be host or device memory (host arrays are staged through the
 * scene's own device buffer).  Asynchronous on `stream`: it returns once
 * the work is enqueued, so a pinned host array must stay unchanged until
 * the stream has passed the call.  A non-finite value is not reported here:
 * the next frame that reads the scene culls all of the scene's triangles
 * and returns PR_ERR_NONFINITE (a later update with finite values clears
 * it).  The caller must not update a scene while a frame that reads it may
 * still be running on another stream, and must order its updates of one
 * scene (keep two scenes to overlap an update with a frame). */
pr_status pr_scene_update(pr_scene *scene, const float *pos, const float *vel, const float *col,
                          void *stream);

/* pr_scene_update for n scenes in one call (for loops that step many
 * scenes every iteration): scene k takes pos[k], vel[k], col[k], DEVICE
 * float32 [V_k][3] arrays (an entry may be NULL to keep that array; pos,
 * vel or col itself may be NULL for none).  pos, vel, col are HOST arrays of
 * n pointers.  Two kernel launches for all the scenes (n <= 4096);
 * asynchronous on `stream`, and a non-finite value is reported by the next
 * frame that reads the scene, exactly as pr_scene_update.
 * PR_ERR_INVALID_ARG for a NULL scene, a host data pointer or n out of
 * range. */
pr_status pr_scene_update_batch(pr_scene *const *scenes, int32_t n, const float *const *pos,
                                const float *const *vel, const float *const *col, void *stream);

void pr_scene_free(pr_scene *scene);

/* Stages (a)-(c) for one view: writes id_out uint32 [H][W] (0xFFFFFFFF =
 * background) and depth_out float32 [H][W] (+inf = background); either may
 * be NULL.  params may be NULL (defaults).  Sec. 3.2 "Bounding" and
 * "Intersection"; bounds of Sec. 4. */
pr_status pr_rasterize(pr_scene *scene, const pr_view *view, const pr_params *params, uint32_t *id_out,
                       float *depth_out, void *stream);

/* Stage (d): deferred Lambert shading with the light interpolated at each
 * pixel's time (Sec. 3.2, "Shading").  id: uint32 [H][W] from
 * pr_rasterize; rgb_out: float32 planar [3][H][W] (0 = background).  When
 * the scene's last pr_rasterize ran the precision form (fp64_retest = 1),
 * so does the shading: a pixel whose FP32 barycentrics are ill-conditioned
 * (a triangle small against its distance) takes its moved triangle,
 * barycentrics and normal from FP64.  The batched calls do the same per
 * their params. */
pr_status pr_shade(pr_scene *scene, const pr_view *view, const uint32_t *id, float *rgb_out, void *stream);

/* Stage (e): adjoint of (d) and of the barycentrics of (c) with the
 * visible ids held fixed.  grad_rgb: float32 planar [3][H][W]; dcol, dpos,
 * dvel: float32 [V][3], ACCUMULATED (+=) by the call; any may be NULL.
 * Not in the paper: the differentiable form of the method. */
pr_status pr_backward(pr_scene *scene, const pr_view *view, const uint32_t *id, const float *grad_rgb,
                      float *dcol, float *dpos, float *dvel, void *stream);

/* One entry of a batched adjoint: the scene and view of a rendered frame,
 * its id buffer, the gradient of the loss w.r.t. its rgb image, and the
 * per-vertex gradient outputs (accumulated; any may be NULL).  DEVICE
 * pointers only. */
typedef struct {
    pr_scene *scene;
    pr_view view;
    const uint32_t *id;        /* [H][W] */
    const float *grad_rgb;     /* [3][H][W] */
    float *dcol, *dpos, *dvel; /* [V][3] of the scene, accumulated (+=) */
} pr_backward_view;

/* Stage (e) for n views in one launch (8x4 pixel blocks of all views in
 * one grid); equal to n calls of pr_backward up to the order of the float
 * additions.  Host pointers are rejected (PR_ERR_INVALID_ARG).  Uses ws
 * only for the view table. */
pr_status pr_backward_batch(pr_workspace *ws, const pr_backward_view *views, int32_t n, void *stream);

/* One entry of a batched call: a scene, a view and its outputs. */
typedef struct {
    pr_scene *scene;
    pr_view view;
    uint32_t *id_out;     /* [H][W] or NULL */
    float *depth_out;     /* [H][W] or NULL */
    float *rgb_out;       /* [3][H][W] or NULL: shade in the same call */
    int32_t tile;         /* 0: params->tile, else 8, 16 or 32 for this view */
    int32_t pad;
} pr_batch_view;

pr_status pr_workspace_create(pr_workspace **out);
void pr_workspace_free(pr_workspace *ws);

/* Stages (a)-(d) for n views of possibly different scenes, sizes and modes
 * as ONE sequence: one bound launch over all triangles, one binning pass
 * over all tiles and one persistent fragment launch per tile size over a
 * global (view, tile) work queue.  Per view, the outputs are bit-identical
 * to pr_rasterize + pr_shade.  Scratch lives in ws. */
pr_status pr_rasterize_batch(pr_workspace *ws, const pr_batch_view *views, int32_t n, const pr_params *params,
                             void *stream);

/* The gradient side of one view of a training frame, at most one of:
 *  - grad_rgb = dL/drgb, float32 [3][H][W];
 *  - target_rgb, float32 [3][H][W], for the L2 loss L = sum (rgb - target)^2
 *    over the view's pixels and channels (then dL/drgb = 2 (rgb - target) is
 *    formed from the frame's own shaded colour inside the adjoint kernel);
 *  - target_u8, uint8 [3][H][W], the same loss against target = value / 255
 *    (an 8-bit image, the form training data usually comes in).
 * dcol, dpos, dvel [V][3] of the view's scene are ACCUMULATED (+=), any may
 * be NULL.  loss: one float, ACCUMULATED (+=) with the view's L (background
 * pixels count with rgb = 0), or NULL; it needs a target.  All DEVICE
 * pointers; the inputs must not overlap the view's outputs.  None of the
 * three: no adjoint for this view.  A view with a gradient entry may leave
 * rgb_out NULL: the colour is formed in registers and not stored. */
typedef struct {
    const float *grad_rgb;
    const float *target_rgb;
    float *dcol, *dpos, *dvel;
    const uint8_t *target_u8;
    float *loss;
} pr_frame_grad;

/* A training frame: pr_rasterize_batch (stages (a)-(d)) followed, in the
 * same sequence and with no host round trip, by stage (e) for every view
 * with a gradient entry (grads: n entries in view order, or NULL).  The
 * adjoint reads the frame's own stage (a) records.  Views with a gradient
 * need a device rgb_out.  When a forward attempt overflows the workspace and
 * is rerun after regrowth, the adjoint of that attempt does nothing, so the
 * gradients are accumulated exactly once per call. */
pr_status pr_frame_batch(pr_workspace *ws, const pr_batch_view *views, int32_t n, const pr_params *params,
                         const pr_frame_grad *grads, void *stream);

/* ---- display step (Sec. 3.1.1, "Display") ----
 * The foveated framebuffer image I_f of a view becomes the display image
 * I_u(x) = I_f(q^-1(x)).  Display pixel (a, b) has its centre at
 * x = ((a + 1/2)/Wd, (b + 1/2)/Hd); views that are not foveated use the
 * identity map.  Under the power map the framebuffer covers a disc around
 * the fovea of the display; display pixels beyond it take the framebuffer's
 * edge values. */
typedef enum {
    PR_UNFOVEATE_MIP_CUBIC = 0, /* MIP pyramid (2x2 box, sizes halved with ceil) sampled tri-linearly at
                                   the level log2(largest stretch of q^-1 at x * max(W/Wd, H/Hd)), each
                                   level with a 3-tap cubic B-spline filter per axis (normalised) */
    PR_UNFOVEATE_PROJECTED = 1  /* the framebuffer pixel holding q^-1(x) and its 5x5 neighbourhood, weighted
                                   by exp(-d^2 / (2 sigma^2)), d = display-pixel distance between x and q of
                                   each pixel centre, normalised by the weights' sum (computed relative
                                   to the nearest sample, so far from the framebuffer they do not all
                                   underflow) */
} pr_unfoveate_method;

typedef struct {
    int32_t method;       /* pr_unfoveate_method */
    int32_t Wd, Hd;       /* display size, 1..16384 */
    float sigma;          /* PROJECTED: filter width in display pixels (> 0) */
} pr_unfoveate_params;

/* rgb: DEVICE planar [3][view.H][view.W] f32 (e.g. a shaded frame); out:
 * DEVICE planar [3][Hd][Wd] f32, written.  view: W, H, mode, fovea and alpha
 * are used.  The MIP pyramid lives in the workspace (grown on demand).
 * Asynchronous on `stream`.  PR_ERR_INVALID_ARG for host pointers or
 * invalid sizes / parameters. */
pr_status pr_unfoveate(pr_workspace *ws, const pr_view *view, const float *rgb, float *out,
                       const pr_unfoveate_params *params, void *stream);

/* One view of a batched display step. */
typedef struct {
    const pr_view *view; /* W, H, mode, fovea, alpha and foveation are used */
    const float *rgb;    /* DEVICE planar [3][view.H][view.W] f32 */
    float *out;          /* DEVICE planar [3][Hd][Wd] f32, written */
    int32_t Wd, Hd;      /* display size, 1..16384 */
} pr_unfoveate_entry;

/* The display step of n views (Sec. 3.1.1, "Display") in one sequence.
 * MIP: one launch per pyramid level over every view that has the level and
 * one over the display pixels of all views, the pyramids side by side in the
 * workspace.  Projected filter: the single-view kernels view after view,
 * each view's q table in the same scratch.  Entry k's out equals that of
 * pr_unfoveate with the same view, rgb, out, Wd, Hd and params->method and
 * sigma, bit for bit; params->Wd and Hd are ignored.  Scratch grows on
 * demand.  The view
 * table goes up through pinned memory of the workspace: a call first waits
 * for the previous batch call's table copy (not for its kernels).
 * Asynchronous on `stream`.  PR_ERR_INVALID_ARG, nothing launched, for
 * n < 0, entries null with n > 0, or any entry that pr_unfoveate refuses. */
pr_status pr_unfoveate_batch(pr_workspace *ws, const pr_unfoveate_entry *entries, int32_t n,
                             const pr_unfoveate_params *params, void *stream);

/* Captures the same sequence into a CUDA graph (after one eager run that
 * sizes every buffer) and replays it with pr_graph_launch.  The views and
 * their buffers must stay valid and unchanged in shape while the graph
 * lives; their contents may change between launches.  The graph keeps its
 * own copy of the view table (poses, intrinsics, modes, output pointers as
 * given at capture) and replays that; it shares the workspace's scratch, so
 * replays and other calls on the same workspace must not overlap on the
 * GPU.  A later call that regrows the workspace makes the graph stale:
 * pr_graph_launch then returns PR_ERR_INVALID_ARG without launching, and the
 * graph must be captured again.  pr_graph_launch returns after the replay's
 * status has been read. */
typedef struct pr_graph pr_graph;
pr_status pr_graph_capture_batch(pr_workspace *ws, const pr_batch_view *views, int32_t n,
                                 const pr_params *params, void *stream, pr_graph **out);
/* The same for a training frame (pr_frame_batch): forward, loss gradient and
 * adjoint replayed as one graph.  Gradient outputs accumulate on every
 * replay (zero them between replays if a fresh gradient is wanted); a replay
 * whose forward overflows skips the adjoint and pr_graph_launch returns
 * PR_ERR_OVERFLOW (an eager call then regrows the workspace; capture again). */
pr_status pr_graph_capture_frame(pr_workspace *ws, const pr_batch_view *views, int32_t n,
                                 const pr_params *params, const pr_frame_grad *grads, void *stream,
                                 pr_graph **out);
pr_status pr_graph_launch(pr_graph *g, void *stream);
/* The two halves of pr_graph_launch, for a frame loop that does not wait on
 * the host after every frame: pr_graph_enqueue launches one replay on
 * stream and returns at once (PR_ERR_INVALID_ARG, nothing launched, for a
 * stale graph); pr_graph_status returns the status of the graph's last
 * replay and fills the workspace statistics, and may be called only once the
 * stream has passed that replay (after a synchronisation the caller makes).
 * Each graph keeps its own copy of its replay's status words, so a loop may
 * read one graph's status while a replay of another graph on the same
 * workspace runs (stage times, when captured, are the workspace's and belong
 * to the last replay).  Replays of graphs that share a workspace must not
 * overlap on the GPU.  pr_graph_free waits for the device to finish. */
pr_status pr_graph_enqueue(pr_graph *g, void *stream);
pr_status pr_graph_status(pr_graph *g);
void pr_graph_free(pr_graph *g);

/* pr_rasterize without allocating: stages (a)-(c) of one view, with every
 * scratch buffer carved from a fixed 64 MiB array that the library keeps in
 * device memory (a file-scope __device__ array, held by every GPU that loads
 * the library until the process exits).  The paper has no counterpart; this
 * entry point exists for callers that may not allocate device memory -- a
 * real-time frame loop in which cudaMalloc/cudaFree would synchronise the
 * device and stall a frame, or a host that owns all GPU memory up front and
 * gives libraries none.
 * pos, vel, col: DEVICE float32 [V][3]; tri: DEVICE int32 [T][3]; id_out
 * uint32 [H][W] and depth_out float32 [H][W]: DEVICE buffers (either may be
 * NULL).  Host pointers are rejected (PR_ERR_INVALID_ARG): staging them
 * would need allocations.  view and params are validated as for
 * pr_rasterize, except that fp64_retest must be 0 (the re-test's flag
 * buffers are not part of the array): fp64_retest = 1 returns
 * PR_ERR_INVALID_ARG.
 * Limits: a frame whose fixed scratch (48 V + 276 T bytes, about 52 bytes
 * per tile, 8 bytes per pixel and the scans' state) does not fit the 64 MiB
 * returns PR_ERR_INVALID_ARG; one whose bins do not fit what is left (20
 * bytes per bin entry) returns PR_ERR_OVERFLOW, whether that is known before
 * the launch or found by the binning kernels.  No buffer grows and nothing
 * is retried.  A bounded device-side wait that ran out returns
 * PR_ERR_TIMEOUT.
 * The first call on a device looks up the array's device address on that
 * device (with it current).
 * Every call waits for its stream before it returns (it reads the frame's
 * status word back).  All calls share the array and it keeps the last
 * call's contents (each call clears what must start at zero); calls that
 * overlap on the GPU -- other streams or other host threads -- race on it
 * and must be serialised.
 * Output equals pr_rasterize with the same arguments. */
pr_status pr_rasterize_noalloc(const float *pos, const float *vel, const float *col, const int32_t *tri,
                               int64_t V, int64_t T, const pr_view *view, const pr_params *params,
                               uint32_t *id_out, float *depth_out, void *stream);

/* Counters of the last rasterize call made with this scene / workspace. */
pr_status pr_scene_stats(const pr_scene *scene, pr_stats *out);
pr_status pr_workspace_stats(const pr_workspace *ws, pr_stats *out);

/* Per-triangle bound of the last pr_rasterize call on this scene (stage
 * (a) output, for tests of conservativeness): pix_box int32 [T][4] =
 * inclusive framebuffer pixel box (i0, j0, i1, j1), empty when i0 > i1;
 * t_range float32 [T][2] = [t_min, t_max]. */
pr_status pr_debug_bounds(const pr_scene *scene, int32_t *pix_box, float *t_range);

/* Half-planes of the per-triangle bound of the last pr_rasterize call on
 * this scene (stage (a) output, for tests of conservativeness): hp float32
 * [T][8][4], slot h = (nx, ny, c, unused), the region is where
 * nx x + ny y + c <= 0; info int32 [T]: bits 0-7 the number of slots in use,
 * bit 8 set when they are framebuffer lines in unit framebuffer coordinates
 * u (the Simple and Recursive foveation bounds of Sec. 4.1.1-4.1.2), clear
 * when they bound the display region in display coordinates x (Sec. 4.2).
 * Culled triangles have no half-planes.  Synchronises the device. */
pr_status pr_debug_halfplanes(const pr_scene *scene, float *hp, int32_t *info);

/* Host evaluation of the stage (a) catch-up interval for one triangle (the
 * Zenon bound of Sec. 4.2.4): S, E float [3][3] camera-space vertices at
 * t = 0 and t = 1; writes [t_min, t_max] and returns 1, or returns 0 when
 * the rolling scan never meets the triangle.  For unit tests. */
int32_t pr_debug_catch_interval(const pr_view *view, const float *S, const float *E, float *t_out);

/* Failure detection of the single-pass scan's bounded wait, for tests: runs
 * a two-tile scan as one block whose predecessor tile never runs, so its
 * look-back wait runs out (after a short limit of polls).  Returns
 * PR_ERR_TIMEOUT when the kernel reported the timeout and finished (the
 * expected outcome; the context stays usable), PR_OK if it did not.  It
 * allocates and frees about 130 KB of device memory. */
pr_status pr_debug_scan_timeout(void *stream);

/* Measures the FP32 fused multiply-add throughput of the current device
 * (TFLOP/s, best of three timed launches of independent FMA chains on every
 * SM, after one warm-up launch) on stream; it allocates and frees a 4 KB
 * buffer.  The paper has no counterpart: it cross-checks the peak against
 * which the fragment stage's ALU roofline is reported.  tflops_out: host
 * pointer, written. */
pr_status pr_measure_fp32_peak(void *stream, double *tflops_out);

const char *pr_status_string(pr_status s);
int32_t pr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PR_H */
