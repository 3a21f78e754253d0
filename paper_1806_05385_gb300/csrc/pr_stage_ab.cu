// pr_stage_ab.cu -- scene upload, stage (a) bounds and stage (b) tile binning.
//
// Stage (a) follows Sec. 3.2 ("Bounding") and Sec. 4: each triangle becomes
// a "space-time triangle" of six camera-space vertices (start and end of the
// frame), and a 2D region is found that holds every display location the
// triangle can cover at the time the rolling scan shows that location.  The
// region is kept in display coordinates (convex hull half-planes plus the
// time strip of the catch-up interval), where it is exact and convex; the
// foveation warp is applied to the framebuffer tiles instead (their display
// images), and to the region only to find the range of framebuffer pixels.
#include <algorithm>

#include "pr_bound.cuh"
#include "pr_launch.h"

namespace pr {

// ---------------------------------------------------------------- scene

// The scene in device memory: a vertex is one 32-byte record (two float4:
// position and velocity, px py pz vx | vy vz 0 0), so the gathers of stage
// (a), of the shading fallback and of the FP64 re-test take one sector per
// vertex; colours are one float4 per vertex and a triangle's indices one
// int4, so the shading kernels gather a visible triangle with one index
// load and three colour loads.
// which: 0 positions, 1 velocities, 2 colours ([V][3] each) into the records.
__global__ void k_scene_set(const float *__restrict__ src, int which, long long V, float4 *__restrict__ vtx,
                            float4 *__restrict__ col4)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= V)
        return;
    const float x = src[3 * k], y = src[3 * k + 1], z = src[3 * k + 2];
    if (which == 0) {
        float4 a = vtx[2 * k];
        a.x = x;
        a.y = y;
        a.z = z;
        vtx[2 * k] = a;
    } else if (which == 1) {
        vtx[2 * k].w = x;
        vtx[2 * k + 1] = make_float4(y, z, 0.f, 0.f);
    } else {
        col4[k] = make_float4(x, y, z, 0.f);
    }
}

__global__ void k_scene_pack(const float *__restrict__ pos, const float *__restrict__ vel,
                             const float *__restrict__ col, long long V, float4 *__restrict__ vtx,
                             float4 *__restrict__ col4)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= V)
        return;
    vtx[2 * k] = make_float4(pos[3 * k], pos[3 * k + 1], pos[3 * k + 2], vel[3 * k]);
    vtx[2 * k + 1] = make_float4(vel[3 * k + 1], vel[3 * k + 2], 0.f, 0.f);
    col4[k] = make_float4(col[3 * k], col[3 * k + 1], col[3 * k + 2], 0.f);
}

cudaError_t launch_scene_set(const float *src, int which, long long V, float4 *vtx, float4 *col4, cudaStream_t st)
{
    if (V > 0)
        k_scene_set<<<(unsigned)((V + 255) / 256), 256, 0, st>>>(src, which, V, vtx, col4);
    return cudaGetLastError();
}

__global__ void k_scene_check(const float4 *__restrict__ vtx, const float4 *__restrict__ col4, long long V,
                              unsigned *status)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= V)
        return;
    const float4 a = vtx[2 * k], b = vtx[2 * k + 1], c = col4[k];
    const bool ok = isfinite(a.x) && isfinite(a.y) && isfinite(a.z) && isfinite(a.w) && isfinite(b.x) &&
                    isfinite(b.y) && isfinite(c.x) && isfinite(c.y) && isfinite(c.z);
    if (!ok)
        atomicOr(status, ST_NONFINITE);
}

// Batched scene update: the statuses are cleared, then every vertex of every
// scene of the chunk takes its new arrays and is checked (blockIdx.y: scene).
struct SceneUpdateChunk {
    SceneUpdate u[kSceneUpdateChunk];
    int n;
};

__global__ void k_scene_status_clear(const SceneUpdateChunk c)
{
    if ((int)threadIdx.x < c.n)
        *c.u[threadIdx.x].status = 0u;
}

__global__ void k_scene_update_batch(const SceneUpdateChunk c)
{
    const SceneUpdate &u = c.u[blockIdx.y];
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= u.V)
        return;
    float4 a = u.vtx[2 * k], b = u.vtx[2 * k + 1], cl = u.col4[k];
    if (u.pos) {
        a.x = u.pos[3 * k];
        a.y = u.pos[3 * k + 1];
        a.z = u.pos[3 * k + 2];
    }
    if (u.vel) {
        a.w = u.vel[3 * k];
        b = make_float4(u.vel[3 * k + 1], u.vel[3 * k + 2], 0.f, 0.f);
    }
    if (u.col)
        cl = make_float4(u.col[3 * k], u.col[3 * k + 1], u.col[3 * k + 2], 0.f);
    u.vtx[2 * k] = a;
    u.vtx[2 * k + 1] = b;
    u.col4[k] = cl;
    const bool ok = isfinite(a.x) && isfinite(a.y) && isfinite(a.z) && isfinite(a.w) && isfinite(b.x) &&
                    isfinite(b.y) && isfinite(cl.x) && isfinite(cl.y) && isfinite(cl.z);
    if (!ok)
        atomicOr(u.status, ST_NONFINITE);
}

cudaError_t launch_scene_update_batch(const SceneUpdate *u, int n, cudaStream_t st)
{
    for (int c0 = 0; c0 < n; c0 += kSceneUpdateChunk) {
        SceneUpdateChunk c;
        c.n = std::min(kSceneUpdateChunk, n - c0);
        long long vmax = 0;
        for (int k = 0; k < c.n; ++k) {
            c.u[k] = u[c0 + k];
            vmax = std::max(vmax, c.u[k].V);
        }
        k_scene_status_clear<<<1, kSceneUpdateChunk, 0, st>>>(c);
        if (vmax > 0)
            k_scene_update_batch<<<dim3((unsigned)((vmax + 255) / 256), (unsigned)c.n), 256, 0, st>>>(c);
    }
    return cudaGetLastError();
}

__global__ void k_scene_idx(const int *__restrict__ tri, long long T, long long V, int4 *__restrict__ tri4,
                            Counters *cnt)
{
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= T)
        return;
    const int a = tri[3 * k], b = tri[3 * k + 1], c = tri[3 * k + 2];
    const bool ok = a >= 0 && a < V && b >= 0 && b < V && c >= 0 && c < V;
    // an invalid triangle becomes the degenerate (0, 0, 0), so no kernel that
    // runs before the host reads the status gathers outside the vertices
    tri4[k] = ok ? make_int4(a, b, c, 0) : make_int4(0, 0, 0, 0);
    if (!ok)
        atomicOr(&cnt->status, ST_BAD_INDEX);
}

cudaError_t launch_scene_pack(const float *pos, const float *vel, const float *col, long long V, float4 *vtx,
                              float4 *col4, cudaStream_t st)
{
    if (V > 0)
        k_scene_pack<<<(unsigned)((V + 255) / 256), 256, 0, st>>>(pos, vel, col, V, vtx, col4);
    return cudaGetLastError();
}

cudaError_t launch_scene_check(const float4 *vtx, const float4 *col4, long long V, unsigned *status, cudaStream_t st)
{
    if (V > 0)
        k_scene_check<<<(unsigned)((V + 255) / 256), 256, 0, st>>>(vtx, col4, V, status);
    return cudaGetLastError();
}

cudaError_t launch_scene_idx(const int *tri, long long T, long long V, int4 *tri4, Counters *cnt, cudaStream_t st)
{
    if (T > 0)
        k_scene_idx<<<(unsigned)((T + 255) / 256), 256, 0, st>>>(tri, T, V, tri4, cnt);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- tiles

// Pixel-centre box of tile lt of view v in unit framebuffer coordinates,
// computed with the same rounding as pixel_ray.
__device__ __forceinline__ void tile_pixel_box(const ViewDev &v, long long lt, float &u0, float &u1, float &w0,
                                               float &w1)
{
    const int ty = (int)lt / v.tiles_x, tx = (int)lt - ty * v.tiles_x;
    const int i0 = tx * v.S, i1 = min(v.W, i0 + v.S) - 1;
    const int j0 = ty * v.S, j1 = min(v.H, j0 + v.S) - 1;
    u0 = __fdiv_rn((float)i0 + 0.5f, (float)v.W);
    u1 = __fdiv_rn((float)i1 + 0.5f, (float)v.W);
    w0 = __fdiv_rn((float)j0 + 0.5f, (float)v.H);
    w1 = __fdiv_rn((float)j1 + 0.5f, (float)v.H);
}

// Display box of every framebuffer tile: the box of its pixel centres, or
// for foveated views the box of their image under q.
__device__ __forceinline__ float4 tile_display_box(const ViewDev *views, int nviews, const long long *tile_offs,
                                                   long long g)
{
    const ViewDev &v = views[find_view(tile_offs, nviews, g)];
    float u0, u1, w0, w1;
    tile_pixel_box(v, g - v.tile_off, u0, u1, w0, w1);
    float4 b;
    if (is_foveated(v.mode))
        b = fov_image_box(u0, u1, w0, w1, make_float2(v.fx, v.fy), v.alpha, v.p_lut, v.p_n);
    else
        b = make_float4(u0, u1, w0, w1);
    const float e = kEpsDisp;
    return make_float4(b.x - e, b.y + e, b.z - e, b.w + e);
}

// ---------------------------------------------------------------- bound

// Result of stage (a) for one triangle.  The half-planes sit in fixed slots
// (kHpEdge + 0..2: edges of the triangle at t_min, kHpMotion + 0..1: across
// its motion, kHpStrip + 0..1: the time strip) so that they stay in
// registers; hmask marks the slots in use.
constexpr int kHpEdge = 0, kHpMotion = 3, kHpStrip = 5;
struct Bound {
    float xmin, xmax, ymin, ymax;  // display box
    float tmin, tmax;              // catch-up interval (0, 0 when not rolling)
    float4 hp[kMaxHp];             // outside iff a x + b y + c > 0
    unsigned hmask;
    int i0, i1, j0, j1;            // framebuffer pixel box (inclusive)
    bool culled;
};

__device__ __forceinline__ float3 lerp_pt(float3 S, float3 D, float t)
{
    return make_float3(fmaf(t, D.x, S.x), fmaf(t, D.y, S.y), fmaf(t, D.z, S.z));
}

// Half-plane with unit normal n that holds the points q[0..nq): n . x <= the
// largest n . q[k], grown by eps.
template <int N>
__device__ __forceinline__ float4 support_halfplane(float2 n, const float2 (&q)[N], int nq, float eps)
{
    float c = -INFINITY;
#pragma unroll
    for (int k = 0; k < N; ++k)
        if (k < nq)
            c = fmaxf(c, fmaf(n.x, q[k].x, n.y * q[k].y));
    return make_float4(n.x, n.y, -c - eps, 0.f);
}

// Framebuffer box that holds q^-1 of a display region R (Sec. 3.1.1: q^-1
// is radial about the fovea f with radius map p^-1).  pts[0..n) span at
// least the angles of R about f and reach at least its largest distance
// from f; rlo is a lower bound of the distance from f to R, used when f is
// outside R.  The preimage then lies in the annular sector of those angles
// and of the radii p^-1 of the nearest and farthest distance.
template <int N>
__device__ __forceinline__ float4 fov_sector_preimage(const float2 (&pts)[N], int n, float2 f, float inv_alpha,
                                                      float eps, bool f_inside, float rlo, const float *lut = nullptr,
                                                      int lut_n = 0)
{
    const SampledP sp{lut, lut_n};
    float rmax = 0.f;
#pragma unroll
    for (int k = 0; k < N; ++k)
        if (k < n) {
            const float2 w = f2sub(pts[k], f);
            rmax = fmaxf(rmax, sqrtf(w.x * w.x + w.y * w.y));
        }
    rmax += eps;
    const float kD1 = powf(kSqrt2, 1.f - inv_alpha);
    const float rho1 = (lut ? sp.pinv(rmax) : kD1 * powf(rmax, inv_alpha)) * (1.f + 1e-5f) + 1e-6f;
    const float rmin = f_inside ? 0.f : fmaxf(0.f, rlo - eps);
    if (rmin <= 0.f)
        return sector_box(f, make_float2(1.f, 0.f), make_float2(1.f, 0.f), 0.f, rho1, true);
    const float rho0 = (lut ? sp.pinv(rmin) : kD1 * powf(rmin, inv_alpha)) * (1.f - 1e-5f);
    // f lies outside the convex hull of the points: their directions from
    // f span less than half a turn, and one sweep finds the two extremes
    float2 a = f2sub(pts[0], f), b = a;
#pragma unroll
    for (int k = 1; k < N; ++k)
        if (k < n) {
            const float2 w = f2sub(pts[k], f);
            if (cross2(a, w) < 0.f)
                a = w;
            if (cross2(b, w) > 0.f)
                b = w;
        }
    const float la = sqrtf(a.x * a.x + a.y * a.y), lb = sqrtf(b.x * b.x + b.y * b.y);
    a = make_float2(a.x / la, a.y / la);
    b = make_float2(b.x / lb, b.y / lb);
    // the region grown by eps spans a little more angle: asin(eps / r)
    a = rot_small(a, -(eps / fmaxf(la, eps) + 1e-6f));
    b = rot_small(b, eps / fmaxf(lb, eps) + 1e-6f);
    if (cross2(a, b) <= 0.f)  // span reached half a turn: give up on angles
        return sector_box(f, a, b, 0.f, rho1, true);
    return sector_box(f, a, b, rho0, rho1, false);
}

// Triangles that reach the near plane (Sec. 4.2.2): the display box of the
// points in front of it and of the crossings of all segments between the
// space-time vertices (loops unrolled, so the points stay in registers).
__device__ __forceinline__ void near_plane_box(const ViewDev &v, const float3 (&P)[6], int np, float &xmin,
                                               float &xmax, float &ymin, float &ymax)
{
    xmin = INFINITY;
    xmax = -INFINITY;
    ymin = INFINITY;
    ymax = -INFINITY;
#pragma unroll
    for (int a = 0; a < 6; ++a) {
        if (a < np && P[a].z >= v.z_near) {
            const float2 q = project(v, P[a]);
            xmin = fminf(xmin, q.x);
            xmax = fmaxf(xmax, q.x);
            ymin = fminf(ymin, q.y);
            ymax = fmaxf(ymax, q.y);
        }
#pragma unroll
        for (int b = a + 1; b < 6; ++b) {
            const float za = P[a].z - v.z_near, zb = P[b].z - v.z_near;
            if (b < np && (za < 0.f) != (zb < 0.f)) {
                const float s = za / (za - zb);
                const float2 q = project(
                    v, make_float3(fmaf(s, P[b].x - P[a].x, P[a].x), fmaf(s, P[b].y - P[a].y, P[a].y), v.z_near));
                xmin = fminf(xmin, q.x);
                xmax = fmaxf(xmax, q.x);
                ymin = fminf(ymin, q.y);
                ymax = fmaxf(ymax, q.y);
            }
        }
    }
}

// q^-1 (display -> framebuffer): radial about the fovea with p^-1(d) =
// D (d/D)^(1/alpha), or the inverse of the view's sampled p.
__device__ __forceinline__ float2 fov_inverse(float2 x, float2 f, float inv_alpha, const float *lut = nullptr,
                                              int lut_n = 0)
{
    const float ex = x.x - f.x, ey = x.y - f.y, r = sqrtf(ex * ex + ey * ey);
    float s;
    if (lut) {
        const SampledP sp{lut, lut_n};
        s = r > 0.f ? sp.pinv(r) / r : 0.f;
    } else {
        s = r > 0.f ? powf(r * (1.f / kSqrt2), inv_alpha - 1.f) : 0.f;
    }
    return make_float2(fmaf(ex, s, f.x), fmaf(ey, s, f.y));
}

// Clips the convex polygon in[0..n) by a x + b y + c <= 0; returns the new size (<= cap).
__device__ __forceinline__ int clip_polygon(const float2 *in, int n, float4 h, float2 *out, int cap)
{
    int m = 0;
    for (int i = 0; i < n; ++i) {
        const float2 p = in[i], q = in[i + 1 < n ? i + 1 : 0];
        const float dp = fmaf(h.x, p.x, fmaf(h.y, p.y, h.z)), dq = fmaf(h.x, q.x, fmaf(h.y, q.y, h.z));
        if (dp <= 0.f && m < cap)
            out[m++] = p;
        if (((dp < 0.f && dq > 0.f) || (dp > 0.f && dq < 0.f)) && m < cap) {
            const float t = dp / (dp - dq);
            out[m++] = make_float2(fmaf(t, q.x - p.x, p.x), fmaf(t, q.y - p.y, p.y));
        }
    }
    return m;
}

// Upper bound of n . u over the framebuffer preimage u = q^-1(y) of the
// display segment a-b (|n| = 1).  q^-1 keeps the direction from the fovea f
// and maps the distance r to p^-1(r), so the preimage lies in the annular
// sector between the directions of a and b (a segment that misses f spans
// less than half a turn) with radii p^-1(r_min) .. p^-1(r_max), r_min and
// r_max the nearest and farthest distances from f to the segment.  A linear
// function peaks over that sector at one of its four corners or, when n
// points between the two directions, on its outer arc.  The radii are
// widened by a relative 1e-5 for FP32 rounding.
constexpr int kFovPieces = 16;
__device__ __forceinline__ float fov_pinv_r(float r, float inv_alpha, const float *lut, int lut_n)
{
    if (lut) {
        const SampledP sp{lut, lut_n};
        return sp.pinv(r);
    }
    return r > 0.f ? kSqrt2 * powf(r * (1.f / kSqrt2), inv_alpha) : 0.f;
}
__device__ float sector_support(float2 a, float2 b, float2 f, float2 n, float inv_alpha, const float *lut, int lut_n)
{
    const float2 pa = make_float2(a.x - f.x, a.y - f.y), pb = make_float2(b.x - f.x, b.y - f.y);
    const float ra = sqrtf(pa.x * pa.x + pa.y * pa.y), rb = sqrtf(pb.x * pb.x + pb.y * pb.y);
    const float2 sg = make_float2(pb.x - pa.x, pb.y - pa.y);
    const float l2 = sg.x * sg.x + sg.y * sg.y;
    float tp = l2 > 0.f ? -(pa.x * sg.x + pa.y * sg.y) / l2 : 0.f;
    tp = fminf(fmaxf(tp, 0.f), 1.f);
    const float cx = fmaf(tp, sg.x, pa.x), cy = fmaf(tp, sg.y, pa.y);
    const float rmin = sqrtf(cx * cx + cy * cy), rmax = fmaxf(ra, rb);
    const float Rmax = fov_pinv_r(rmax, inv_alpha, lut, lut_n) * (1.f + 1e-5f) + 1e-7f;
    const float base = n.x * f.x + n.y * f.y;
    if (!(rmin > 1e-6f * (1.f + rmax)))  // the segment passes (next to) the fovea: the whole disc
        return base + Rmax;
    const float Rmin = fov_pinv_r(rmin, inv_alpha, lut, lut_n) * (1.f - 1e-5f);
    float best = -INFINITY;
    const float da = (n.x * pa.x + n.y * pa.y) / ra, db = (n.x * pb.x + n.y * pb.y) / rb;
    best = fmaxf(best, da * (da > 0.f ? Rmax : Rmin));
    best = fmaxf(best, db * (db > 0.f ? Rmax : Rmin));
    const float cab = pa.x * pb.y - pa.y * pb.x;
    const float can = pa.x * n.y - pa.y * n.x, cnb = n.x * pb.y - n.y * pb.x;
    if ((cab > 0.f && can >= 0.f && cnb >= 0.f) || (cab < 0.f && can <= 0.f && cnb <= 0.f))
        best = fmaxf(best, Rmax);  // n points into the sector: its outer arc
    return base + best;
}

// The paper's foveated edge bounds (Sec. 4.1).  The region's display
// polygon (its box clipped by its half-planes) is bounded edge by edge in
// the framebuffer: the image under q^-1 of the straight edge x0 -> x1 is a
// curve, and the bounding line has the edge's own direction (Simple) or the
// direction of the chord between q^-1(x0) and q^-1(x1) (Recursive), pushed
// out past the farthest point of the curved region along its normal.  The
// paper pushes each line out to its own curve only, which does not hold the
// region when a neighbouring curve bulges past the line under a strong warp;
// here every curve is bounded.  The paper finds each farthest point by a
// ternary search over the edge parameter, which assumes one maximum per
// edge; under alpha = 3 near the fovea, where q^-1 stretches without bound,
// that search missed pixels, so each curve's support is bounded instead
// (sector_support over kFovPieces pieces), and the line gets half a pixel
// of margin.  Writes the framebuffer half-planes to out (at most kMaxHp);
// returns their number (0 when the polygon has more edges than that) and
// their box.
struct PaperFov {
    int n;
    float4 fb;
};
__device__ __forceinline__ PaperFov paper_fov_bound(const ViewDev &v, const float4 *hps, unsigned hmask, float xmin,
                                                 float xmax, float ymin, float ymax, float4 *out)
{
    PaperFov r;
    r.n = 0;
    r.fb = make_float4(1.f, 0.f, 1.f, 0.f);  // empty
    float2 A[16], Bv[16];
    A[0] = make_float2(xmin, ymin);
    A[1] = make_float2(xmax, ymin);
    A[2] = make_float2(xmax, ymax);
    A[3] = make_float2(xmin, ymax);
    int n = 4;
    for (int h = 0; h < kMaxHp; ++h)
        if (hmask & (1u << h)) {
            n = clip_polygon(A, n, hps[h], Bv, 16);
            for (int k = 0; k < n; ++k)
                A[k] = Bv[k];
        }
    // drop repeated vertices (zero-length edges)
    int m = 0;
    for (int k = 0; k < n; ++k) {
        const float2 p = A[k], q = m > 0 ? A[m - 1] : A[n - 1];
        if (m == 0 ? true : (fabsf(p.x - q.x) + fabsf(p.y - q.y) > 1e-9f))
            A[m++] = p;
    }
    if (m > 1 && fabsf(A[0].x - A[m - 1].x) + fabsf(A[0].y - A[m - 1].y) <= 1e-9f)
        --m;
    if (m < 3 || m > kMaxHp)
        return r;
    const float2 f = make_float2(v.fx, v.fy);
    const float margin = 0.5f / (float)max(v.W, v.H) + 1e-6f;
    const float px = (float)max(v.W, v.H);
    for (int k = 0; k < m; ++k) {
        const float2 x0 = A[k], x1 = A[k + 1 < m ? k + 1 : 0];
        float2 d = make_float2(x1.x - x0.x, x1.y - x0.y);
        if (v.fov_bound == PR_FOV_RECURSIVE) {
            const float2 a = fov_inverse(x0, f, v.inv_alpha, v.p_lut, v.p_n),
                         b = fov_inverse(x1, f, v.inv_alpha, v.p_lut, v.p_n);
            const float2 c = make_float2(b.x - a.x, b.y - a.y);
            if (c.x * c.x + c.y * c.y > 1e-20f)
                d = c;
        }
        const float len = sqrtf(d.x * d.x + d.y * d.y);
        const float2 nrm = make_float2(d.y / len, -d.x / len);  // outward for the counter-clockwise polygon
        // the line must hold the whole curved region, not only its own edge's
        // image (under a strong warp a neighbouring curve can bulge past it):
        // the largest support along the normal over every curved edge,
        // bounded rigorously over 16 pieces of each edge
        float best = -INFINITY;
        for (int e = 0; e < m; ++e) {
            const float2 y0 = A[e], y1 = A[e + 1 < m ? e + 1 : 0];
            for (int j = 0; j < kFovPieces; ++j) {
                const float s0 = j * (1.f / kFovPieces), s1 = (j + 1) * (1.f / kFovPieces);
                const float2 a = make_float2(fmaf(s0, y1.x - y0.x, y0.x), fmaf(s0, y1.y - y0.y, y0.y));
                const float2 b = make_float2(fmaf(s1, y1.x - y0.x, y0.x), fmaf(s1, y1.y - y0.y, y0.y));
                best = fmaxf(best, sector_support(a, b, f, nrm, v.inv_alpha, v.p_lut, v.p_n));
            }
        }
        out[k] = make_float4(nrm.x, nrm.y, -(best + margin), 0.f);
    }
    // framebuffer box: the viewport clipped by the bounding lines
    A[0] = make_float2(-margin, -margin);
    A[1] = make_float2(1.f + margin, -margin);
    A[2] = make_float2(1.f + margin, 1.f + margin);
    A[3] = make_float2(-margin, 1.f + margin);
    n = 4;
    for (int k = 0; k < m; ++k) {
        n = clip_polygon(A, n, out[k], Bv, 16);
        for (int j = 0; j < n; ++j)
            A[j] = Bv[j];
    }
    r.n = m;
    if (n == 0)
        return r;
    float4 fb = make_float4(INFINITY, -INFINITY, INFINITY, -INFINITY);
    for (int j = 0; j < n; ++j) {
        fb.x = fminf(fb.x, A[j].x);
        fb.y = fmaxf(fb.y, A[j].x);
        fb.z = fminf(fb.z, A[j].y);
        fb.w = fmaxf(fb.w, A[j].y);
    }
    r.fb = fb;
    return r;
}

__device__ __forceinline__ void compute_bound(const ViewDev &v, const float3 S[3], const float3 D[3], Bound &B)
{
    const bool rolling = is_rolling(v.mode), fov = is_foveated(v.mode);
    const float eps = kEpsDisp;
    B.hmask = 0u;
    B.culled = false;
    B.tmin = rolling ? v.t_lo : 0.f;
    B.tmax = rolling ? v.t_hi : 0.f;

    // the relevant space-time points: the triangle at the ends of the time domain
    float3 P[6];
    const int np = rolling && B.tmax != B.tmin ? 6 : 3;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        P[k] = lerp_pt(S[k], D[k], B.tmin);
        P[3 + k] = lerp_pt(S[k], D[k], B.tmax);
    }
    // frustum culling against the near plane and the four side planes
    bool all_near = true, all_l = true, all_r = true, all_t = true, all_b = true, any_near = false;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        if (k >= np)
            break;
        const float3 p = P[k];
        const float mx = 1e-6f * (fabsf(p.x) + v.tan_x * fabsf(p.z)) + 1e-30f;
        const float my = 1e-6f * (fabsf(p.y) + v.tan_y * fabsf(p.z)) + 1e-30f;
        all_near &= p.z < v.z_near;
        any_near |= p.z < v.z_near * (1.f + 1e-6f);
        all_l &= p.x + v.tan_x * p.z < -mx;
        all_r &= v.tan_x * p.z - p.x < -mx;
        all_t &= p.y + v.tan_y * p.z < -my;
        all_b &= v.tan_y * p.z - p.y < -my;
    }
    if (all_near || all_l || all_r || all_t || all_b) {
        B.culled = true;
        return;
    }
    // foveated: the framebuffer covers only part of the display.  The
    // projected time-domain points bound the display region (Sec. 4.2.2), so
    // the sector preimage of their box bounds the triangle's pixels; if that
    // pixel box is empty the triangle leaves before the rest of the bound.
    if (fov && !any_near) {
        float bx0 = INFINITY, bx1 = -INFINITY, by0 = INFINITY, by1 = -INFINITY;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            if (k >= np)
                break;
            const float2 x = project(v, P[k]);
            bx0 = fminf(bx0, x.x);
            bx1 = fmaxf(bx1, x.x);
            by0 = fminf(by0, x.y);
            by1 = fmaxf(by1, x.y);
        }
        const float m = eps * fmaxf(1.f, fmaxf(fmaxf(fabsf(bx0), fabsf(bx1)), fmaxf(fabsf(by0), fabsf(by1))));
        bx0 -= m;
        bx1 += m;
        by0 -= m;
        by1 += m;
        const float2 f = make_float2(v.fx, v.fy);
        const float dbx = fmaxf(fmaxf(bx0 - f.x, f.x - bx1), 0.f), dby = fmaxf(fmaxf(by0 - f.y, f.y - by1), 0.f);
        const float rlo = sqrtf(dbx * dbx + dby * dby);
        const float2 corners[4] = {make_float2(bx0, by0), make_float2(bx1, by0), make_float2(bx1, by1),
                                   make_float2(bx0, by1)};
        const float4 fb = fov_sector_preimage(corners, 4, f, v.inv_alpha, 2.f * eps, rlo <= 2.f * eps, rlo, v.p_lut,
                                              v.p_n);
        // pixel centres inside the preimage box, 1/100 pixel of slack (as below)
        const float fi0 = ceilf(fb.x * v.W - 0.51f), fi1 = floorf(fb.y * v.W - 0.49f);
        const float fj0 = ceilf(fb.z * v.H - 0.51f), fj1 = floorf(fb.w * v.H - 0.49f);
        if (fmaxf(fi0, 0.f) > fminf(fi1, (float)(v.W - 1)) || fmaxf(fj0, 0.f) > fminf(fj1, (float)(v.H - 1))) {
            B.culled = true;
            return;
        }
    }

    float2 Q[6];  // display points of the region (projected space-time vertices)
    int nq = 0;
    bool use_hull = v.bound != PR_BOUND_QUAD && v.bound != PR_BOUND_TRIVIAL;
    bool strip = false;
    float xmin, xmax, ymin, ymax;
    if (any_near) {
        near_plane_box(v, P, np, xmin, xmax, ymin, ymax);
        use_hull = false;
    } else {
        float tmin = B.tmin, tmax = B.tmax;
        if (rolling) {
            if (v.bound == PR_BOUND_ZENON) {
                if (!catch_interval(S, D, v.tan_x, v.tan_y, v.d0, v.d1, v.t_lo, v.t_hi, tmin, tmax)) {
                    B.culled = true;
                    return;
                }
                strip = true;
            } else if (v.bound == PR_BOUND_ADAPTIVE) {
                // Sec. 4.2.3: the times at which the projected space-time
                // vertices are shown bound the times of every covered pixel
                float lo = INFINITY, hi = -INFINITY;
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    if (k >= np)
                        break;
                    const float2 x = project(v, P[k]);
                    const float r = fmaf(x.x, v.d0, x.y * v.d1);
                    lo = fminf(lo, r);
                    hi = fmaxf(hi, r);
                }
                tmin = fmaxf(v.t_lo, lo - kEpsT);
                tmax = fminf(v.t_hi, hi + kEpsT);
                if (!(tmin <= tmax)) {
                    B.culled = true;
                    return;
                }
                strip = true;
            }
            B.tmin = tmin;
            B.tmax = tmax;
        }
        nq = rolling && tmax != tmin ? 6 : 3;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            Q[k] = project(v, lerp_pt(S[k], D[k], tmin));
            Q[3 + k] = project(v, lerp_pt(S[k], D[k], tmax));
        }
        xmin = ymin = INFINITY;
        xmax = ymax = -INFINITY;
#pragma unroll
        for (int k = 0; k < 6; ++k)
            if (k < nq) {
                xmin = fminf(xmin, Q[k].x);
                xmax = fmaxf(xmax, Q[k].x);
                ymin = fminf(ymin, Q[k].y);
                ymax = fmaxf(ymax, Q[k].y);
            }
    }
    const float mx = eps * fmaxf(1.f, fmaxf(fabsf(xmin), fabsf(xmax)));
    const float my = eps * fmaxf(1.f, fmaxf(fabsf(ymin), fabsf(ymax)));
    xmin -= mx;
    xmax += mx;
    ymin -= my;
    ymax += my;
    if (v.bound == PR_BOUND_TRIVIAL) {
        xmin = ymin = -eps;
        xmax = ymax = 1.f + eps;
    }
    if (strip) {
        // the time strip t_min <= d . x <= t_max (covered pixels satisfy t = r(x))
        const float dn = sqrtf(v.d0 * v.d0 + v.d1 * v.d1);
        if (v.d1 == 0.f) {
            xmin = fmaxf(xmin, (B.tmin - kEpsT) / v.d0);
            xmax = fminf(xmax, (B.tmax + kEpsT) / v.d0);
        } else if (v.d0 == 0.f) {
            ymin = fmaxf(ymin, (B.tmin - kEpsT) / v.d1);
            ymax = fminf(ymax, (B.tmax + kEpsT) / v.d1);
        }
        B.hp[kHpStrip] = make_float4(-v.d0 / dn, -v.d1 / dn, (B.tmin - kEpsT) / dn, 0.f);
        B.hp[kHpStrip + 1] = make_float4(v.d0 / dn, v.d1 / dn, -(B.tmax + kEpsT) / dn, 0.f);
        B.hmask |= 3u << kHpStrip;
    }
    // clip to the viewport (every ray's display location lies in [0,1]^2)
    xmin = fmaxf(xmin, -eps);
    ymin = fmaxf(ymin, -eps);
    xmax = fminf(xmax, 1.f + eps);
    ymax = fminf(ymax, 1.f + eps);
    if (!(xmin <= xmax && ymin <= ymax)) {
        B.culled = true;
        return;
    }
    B.xmin = xmin;
    B.xmax = xmax;
    B.ymin = ymin;
    B.ymax = ymax;

    // Sec. 4.2.2: the convex hull of the projected space-time vertices.  Its
    // half-planes are taken as support lines of the points in the three edge
    // directions of the triangle at t_min and the two directions across the
    // triangle's mean motion: for a motion that is a translation these are
    // exactly the hull's edges, otherwise they bound a slightly larger
    // convex region -- still a bound.
    if (use_hull) {
        const float gm = eps * fmaxf(1.f, fmaxf(fmaxf(fabsf(xmin), fabsf(xmax)), fmaxf(fabsf(ymin), fabsf(ymax))));
        const float area = cross2(f2sub(Q[1], Q[0]), f2sub(Q[2], Q[0]));
        if (area != 0.f) {
            const float orient = area > 0.f ? 1.f : -1.f;  // outward normal = orient * (ey, -ex)
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                const float2 p = Q[e], q = Q[(e + 1) % 3];
                const float ex = q.x - p.x, ey = q.y - p.y, l2 = ex * ex + ey * ey;
                if (l2 > 0.f) {
                    const float il = orient / sqrtf(l2);
                    B.hp[kHpEdge + e] = support_halfplane(make_float2(ey * il, -ex * il), Q, nq, gm);
                    B.hmask |= 1u << (kHpEdge + e);
                }
            }
        }
        if (nq == 6) {
            float mvx = 0.f, mvy = 0.f;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                mvx += Q[3 + k].x - Q[k].x;
                mvy += Q[3 + k].y - Q[k].y;
            }
            const float l2 = mvx * mvx + mvy * mvy;
            if (l2 > 0.f) {
                const float il = 1.f / sqrtf(l2);
                const float2 n = make_float2(-mvy * il, mvx * il);
                B.hp[kHpMotion] = support_halfplane(n, Q, nq, gm);
                B.hp[kHpMotion + 1] = support_halfplane(make_float2(-n.x, -n.y), Q, nq, gm);
                B.hmask |= 3u << kHpMotion;
            }
        }
    }

    // framebuffer pixel box
    float u0, u1, w0, w1;
    if (fov) {
        const float2 f = make_float2(v.fx, v.fy);
        // distance from f to the region: at least its distance to the box and
        // to every half-plane it violates
        const float dbx = fmaxf(fmaxf(xmin - f.x, f.x - xmax), 0.f), dby = fmaxf(fmaxf(ymin - f.y, f.y - ymax), 0.f);
        float rlo = sqrtf(dbx * dbx + dby * dby);
#pragma unroll
        for (int h = 0; h < kMaxHp; ++h)
            if (B.hmask & (1u << h))
                rlo = fmaxf(rlo, fmaf(B.hp[h].x, f.x, fmaf(B.hp[h].y, f.y, B.hp[h].z)));
        const bool inside = rlo <= 2.f * eps;
        float4 fb;
        if (use_hull) {
            fb = fov_sector_preimage(Q, nq, f, v.inv_alpha, 2.f * eps, inside, rlo, v.p_lut, v.p_n);
        } else {
            const float2 corners[4] = {make_float2(xmin, ymin), make_float2(xmax, ymin), make_float2(xmax, ymax),
                                       make_float2(xmin, ymax)};
            fb = fov_sector_preimage(corners, 4, f, v.inv_alpha, 2.f * eps, inside, rlo, v.p_lut, v.p_n);
        }
        u0 = fb.x;
        u1 = fb.y;
        w0 = fb.z;
        w1 = fb.w;
    } else {
        u0 = xmin;
        u1 = xmax;
        w0 = ymin;
        w1 = ymax;
    }
    // pixel centres (i + .5)/W inside [u0, u1]; the slack of 1/100 pixel each
    // side covers the FP32 rounding of u W (a few ulps of at most 16384)
    const float fi0 = ceilf(u0 * v.W - 0.51f), fi1 = floorf(u1 * v.W - 0.49f);
    const float fj0 = ceilf(w0 * v.H - 0.51f), fj1 = floorf(w1 * v.H - 0.49f);
    B.i0 = (int)fmaxf(fi0, 0.f);
    B.i1 = (int)fminf(fi1, (float)(v.W - 1));
    B.j0 = (int)fmaxf(fj0, 0.f);
    B.j1 = (int)fminf(fj1, (float)(v.H - 1));
    if (B.i0 > B.i1 || B.j0 > B.j1)
        B.culled = true;
}

// Fragment record layout (6 x float4 per triangle):
//   [0] S0.x S0.y S0.z S1.x   [1] S1.y S1.z S2.x S2.y   [2] S2.z D0.x D0.y D0.z
//   [3] D1.x D1.y D1.z D2.x   [4] xmin xmax ymin ymax   [5] tmin tmax D2.y D2.z
// S = camera-space vertex at t = 0, D = its motion over the frame, the box
// and interval of stage (a).  tbox = (i0 | i1 << 16, j0 | j1 << 16, nhp, depth order
// key of the nearest depth the triangle reaches).  cand = candidate tiles of
// the framebuffer box; the triangles that have some are also appended to
// `binned` (cnt->binned of them), the index space of the binning pass.
__global__ void __launch_bounds__(128, 6) k_bound(const ViewDev *__restrict__ views, int nviews,
                                               const long long *__restrict__ tri_offs, long long ttot,
                                               float4 *__restrict__ rec, float4 *__restrict__ hp,
                                               int4 *__restrict__ tbox, unsigned long long *__restrict__ cand,
                                               int *__restrict__ binned, Counters *cnt)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    // the view of the warp's first triangle by the whole warp (no chain of
    // dependent loads), then each lane steps to its own: a warp's 32
    // triangles meet at most a few view boundaries
    const long long g0 = g - (threadIdx.x & 31);
    if (g0 >= ttot)
        return;  // the whole warp
    int q = find_view_warp(tri_offs, nviews, g0);
    if (g >= ttot)
        return;
    while (q + 1 < nviews && g >= tri_offs[q + 1])
        ++q;
    const ViewDev &v = views[q];
    const int k = (int)(g - v.tri_off);
    const int4 tv = v.tri4[k];
    const int ia = tv.x, ib = tv.y, ic = tv.z;
    float3 S[3], E[3], D[3];
    vertex_start_end(v, ia, S[0], E[0]);
    vertex_start_end(v, ib, S[1], E[1]);
    vertex_start_end(v, ic, S[2], E[2]);
    for (int q = 0; q < 3; ++q)
        D[q] = make_float3(E[q].x - S[q].x, E[q].y - S[q].y, E[q].z - S[q].z);
    Bound B;
    // a scene updated with a non-finite value: every triangle of it is
    // culled (nothing downstream sees its coordinates) and the frame reports it
    const bool bad = v.scene_status && (*v.scene_status & ST_NONFINITE);
    if (bad) {
        B.culled = true;
        const unsigned bm = __activemask();
        if ((threadIdx.x & 31) == __ffs(bm) - 1)
            atomicOr(&cnt->status, ST_NONFINITE);
    } else {
        compute_bound(v, S, D, B);
    }
    float4 *r = rec + g * kRecF4;
    r[0] = make_float4(S[0].x, S[0].y, S[0].z, S[1].x);
    r[1] = make_float4(S[1].y, S[1].z, S[2].x, S[2].y);
    r[2] = make_float4(S[2].z, D[0].x, D[0].y, D[0].z);
    r[3] = make_float4(D[1].x, D[1].y, D[1].z, D[2].x);
    if (B.culled) {
        r[4] = make_float4(INFINITY, -INFINITY, INFINITY, -INFINITY);
        r[5] = make_float4(INFINITY, -INFINITY, D[2].y, D[2].z);
        tbox[g] = make_int4(1, 1, 0, 0);  // the empty box [1, 0] x [1, 0]
        cand[g] = 0ull;
        const unsigned cm = __activemask();  // one atomic per warp
        if ((threadIdx.x & 31) == __ffs(cm) - 1)
            atomicAdd(&cnt->culled, (unsigned long long)__popc(cm));
        return;
    }
    r[4] = make_float4(B.xmin, B.xmax, B.ymin, B.ymax);
    r[5] = make_float4(B.tmin - kEpsT, B.tmax + kEpsT, D[2].y, D[2].z);
    int nhp = 0;
#pragma unroll
    for (int h = 0; h < kMaxHp; ++h)
        if (B.hmask & (1u << h))
            hp[g * kMaxHp + nhp++] = B.hp[h];
    // nearest camera depth the moving triangle reaches (z is linear in t on
    // every vertex): min_k S_k.z + min(0, D_k.z), the sort key of its pairs
    const float near = fminf(fminf(S[0].z + fminf(0.f, D[0].z), S[1].z + fminf(0.f, D[1].z)),
                             S[2].z + fminf(0.f, D[2].z));
    tbox[g] = make_int4(B.i0 | (B.i1 << 16), B.j0 | (B.j1 << 16), nhp, (int)depth_order_key(near));
    cand[g] = (unsigned long long)(B.i1 / v.S - B.i0 / v.S + 1) * (unsigned long long)(B.j1 / v.S - B.j0 / v.S + 1);
    // list the triangle for binning (one atomic per warp; the list order
    // does not matter: every bin is sorted by depth later)
    const unsigned m = __activemask();
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader)
        base = atomicAdd(&cnt->binned, (unsigned long long)__popc(m));
    base = __shfl_sync(m, base, leader);
    binned[base + __popc(m & ((1u << lane) - 1u))] = (int)g;
}

cudaError_t launch_bound(const ViewDev *views, int nviews, const long long *tri_offs, long long ttot, float4 *rec,
                         float4 *hp, int4 *tbox, unsigned long long *cand, int *binned, Counters *cnt, cudaStream_t st)
{
    if (ttot > 0)
        k_bound<<<(unsigned)((ttot + 127) / 128), 128, 0, st>>>(views, nviews, tri_offs, ttot, rec, hp, tbox, cand,
                                                                binned, cnt);
    return cudaGetLastError();
}

// The paper's foveation edge bounds (pr_fov_bound SIMPLE / RECURSIVE), as
// a pass over the stage (a) output of the foveated views that ask for them:
// the display region (box and half-planes) becomes a framebuffer polygon,
// whose half-planes (flag 0x100 in tbox.z) and box replace the sector
// bound's for binning.  Kept out of k_bound so that the default path keeps
// its registers.
__global__ void __launch_bounds__(128) k_paper_fov(const ViewDev *__restrict__ views, int nviews,
                                                   const long long *__restrict__ tri_offs, long long ttot,
                                                   const float4 *__restrict__ rec, float4 *__restrict__ hp,
                                                   int4 *__restrict__ tbox, unsigned long long *__restrict__ cand)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= ttot || cand[g] == 0ull)
        return;
    const ViewDev &v = views[find_view(tri_offs, nviews, g)];
    if (!is_foveated(v.mode) || v.fov_bound == PR_FOV_SECTOR)
        return;
    const int4 tb = tbox[g];
    const float4 box = rec[g * kRecF4 + 4];
    float4 hps[kMaxHp];
    unsigned hmask = 0u;
    for (int h = 0; h < kMaxHp; ++h) {
        hps[h] = hp[g * kMaxHp + h];
        if (h < (tb.z & 0xff))
            hmask |= 1u << h;
    }
    float4 out[kMaxHp];
    const PaperFov pf = paper_fov_bound(v, hps, hmask, box.x, box.y, box.z, box.w, out);
    if (pf.n == 0)
        return;  // more edges than half-plane slots: keep the sector bound
    for (int h = 0; h < pf.n; ++h)
        hp[g * kMaxHp + h] = out[h];
    const float fi0 = ceilf(pf.fb.x * v.W - 0.51f), fi1 = floorf(pf.fb.y * v.W - 0.49f);
    const float fj0 = ceilf(pf.fb.z * v.H - 0.51f), fj1 = floorf(pf.fb.w * v.H - 0.49f);
    const int i0 = (int)fmaxf(fi0, 0.f), i1 = (int)fminf(fi1, (float)(v.W - 1));
    const int j0 = (int)fmaxf(fj0, 0.f), j1 = (int)fminf(fj1, (float)(v.H - 1));
    if (i0 > i1 || j0 > j1) {
        tbox[g] = make_int4(1, 1, 0, tb.w);
        cand[g] = 0ull;
        return;
    }
    tbox[g] = make_int4(i0 | (i1 << 16), j0 | (j1 << 16), pf.n | 0x100, tb.w);
    cand[g] = (unsigned long long)(i1 / v.S - i0 / v.S + 1) * (unsigned long long)(j1 / v.S - j0 / v.S + 1);
}

cudaError_t launch_paper_fov(const ViewDev *views, int nviews, const long long *tri_offs, long long ttot,
                             const float4 *rec, float4 *hp, int4 *tbox, unsigned long long *cand, cudaStream_t st)
{
    if (ttot > 0)
        k_paper_fov<<<(unsigned)((ttot + 127) / 128), 128, 0, st>>>(views, nviews, tri_offs, ttot, rec, hp, tbox,
                                                                    cand);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- binning

// Does the display region of a triangle meet the display box of a tile?
// Box overlap, then every half-plane against the box corner that lies
// deepest inside it.
__device__ __forceinline__ bool tile_meets(const float4 tb, const float4 bb, const float4 *h, int nh)
{
    if (bb.x > tb.y || bb.y < tb.x || bb.z > tb.w || bb.w < tb.z)
        return false;
    // all half-planes are loaded before any is tested (no chain of loads)
    bool out = false;
#pragma unroll
    for (int k = 0; k < kMaxHp; ++k) {
        if (k < nh) {
            const float4 p = h[k];
            const float m = fmaf(p.x, p.x > 0.f ? tb.x : tb.y, fmaf(p.y, p.y > 0.f ? tb.z : tb.w, p.z));
            out |= m > 0.f;
        }
    }
    return !out;
}

// Bins.  Every triangle's framebuffer box spans a rectangle of candidate
// tiles.  The triangles that have candidates are listed in `binned` (by the
// bound pass, m of them) and cand_off is the prefix sum of their counts, so
// candidate pair p belongs to list entry e with cand_off[e] <= p <
// cand_off[e+1].  Warps take the pairs in tasks of consecutive pairs, which
// keeps the work balanced when a few triangles -- near the fovea, where
// q^-1 magnifies, or close to the camera -- span thousands of tiles.
// tile_cnt[tile] = number of triangles whose region meets the tile; every
// hit is appended to the hit list (one atomic per warp) and counted per
// tile (one atomic per distinct tile of a warp).  A bin entry is (depth
// order key of the triangle << 32) | its batch-wide index, so that sorting
// entries sorts by nearest depth.

// Largest e in [0, m) with cand_off[e] <= p for a warp-uniform p, found by
// the whole warp: each step probes 32 evenly spaced offsets of the range
// with one load and keeps the part between the last probe at or below p
// and the next (a 32-ary search: ceil(log32 m) dependent loads).
__device__ __forceinline__ long long warp_owner(const unsigned long long *cand_off, long long m, long long p)
{
    const int lane = threadIdx.x & 31;
    long long lo = 0, hi = m - 1;  // cand_off[lo] <= p; the answer lies in [lo, hi]
    while (hi > lo) {
        const long long span = hi - lo;  // probes lo + 1 .. hi
        const long long idx = span <= 32 ? min(lo + 1 + lane, hi) : lo + 1 + (span - 1) * lane / 31;
        const unsigned le = __ballot_sync(0xffffffffu, (long long)cand_off[idx] <= p);
        if (!le) {
            hi = __shfl_sync(0xffffffffu, idx, 0) - 1;
        } else {
            const int last = 31 - __clz(le);  // probes ascend, so `le` is a prefix of the lanes
            const long long nlo = __shfl_sync(0xffffffffu, idx, last);
            const long long nhi = last < 31 ? __shfl_sync(0xffffffffu, idx, last + 1) - 1 : hi;
            lo = nlo;
            hi = max(nhi, nlo);
        }
    }
    return lo;
}

// The same for one lane's p (a plain binary search): only for pairs that a
// warp's window of 32 list entries does not reach, which needs entries
// without candidates (the paper's foveation bounds can empty a box).
__device__ __forceinline__ long long owner_of(const unsigned long long *cand_off, long long m, long long p)
{
    long long lo = 0, hi = m - 1;
    while (lo < hi) {
        const long long mid = (lo + hi + 1) >> 1;
        if ((long long)cand_off[mid] <= p)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

constexpr int kBinChunks = 8;

// 256 threads, at most 64 registers: four CTAs (32 warps) per SM.  The
// grid is four waves of them (bin_count_grid): the task loop is
// grid-stride, so CTAs that start late take the place of those whose tasks
// ran short, which evens out the end of the pass.
__global__ void __launch_bounds__(256, 4) k_bin(const ViewDev *__restrict__ views, int nviews,
                                             const long long *__restrict__ tri_offs, const int *__restrict__ binned,
                                             const unsigned long long *__restrict__ cand_off,
                                             const float4 *__restrict__ rec, const float4 *__restrict__ hp,
                                             const int4 *__restrict__ tbox, const float4 *__restrict__ tile_box,
                                             unsigned long long *__restrict__ tile_cnt,
                                             unsigned long long *__restrict__ hit_entry,
                                             unsigned *__restrict__ hit_tile, long long cap_pairs, Counters *cnt)
{
    const long long m = (long long)cnt->binned;
    if (m == 0)
        return;
    const long long total = (long long)cand_off[m];
    const int lane = threadIdx.x & 31;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    // Each warp takes tasks of kBinChunks x 32 consecutive candidate pairs.
    // The list entry of the task's first pair comes from a warp-wide 32-ary
    // search; the entries of each chunk's pairs then follow from the offsets
    // of the next 32 entries, loaded with one coalesced read and searched
    // with shuffles (every entry owns at least one pair, so 32 pairs never
    // reach past them).  All lanes run the same iterations (for the shuffles).
    for (long long pt = ((long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * (32 * kBinChunks);
         pt < total; pt += nwarps * (32 * kBinChunks)) {
        long long e0 = warp_owner(cand_off, m, pt);
        // the task's hits: per chunk the ballot, the lane's entry and tile
        unsigned want_c[kBinChunks];
        unsigned long long ent_c[kBinChunks];
        unsigned tile_c[kBinChunks];
#pragma unroll
        for (int c = 0; c < kBinChunks; ++c) {
            want_c[c] = 0u;
            ent_c[c] = 0ull;
            tile_c[c] = 0u;
            const long long pw = pt + 32 * c;
            if (pw >= total)
                continue;  // warp-uniform
            const long long p = pw + lane;
            const long long el = e0 + 1 + lane;
            const unsigned long long o = el <= m ? cand_off[el] : ~0ull;
            // every lane takes part in every shuffle; the fallback search
            // (no warp operations) runs after them
            int k = 0;  // offsets of the window at or below p
            for (int sstep = 16; sstep > 0; sstep >>= 1) {
                const unsigned long long probe = __shfl_sync(0xffffffffu, o, k + sstep - 1);
                if (probe <= (unsigned long long)p)
                    k += sstep;
            }
            const bool beyond = __shfl_sync(0xffffffffu, o, 31) <= (unsigned long long)p;
            const long long e = beyond ? owner_of(cand_off, m, p) : e0 + k;
            e0 = __shfl_sync(0xffffffffu, e, 31);  // owners ascend with p
            bool hit = false, ok_tile = true;
            long long tile = -1;
            unsigned key = 0u;
            long long g = 0;
            if (p < total) {
                g = binned[e];
                const int4 tb = tbox[g];
                key = (unsigned)tb.w;
                const ViewDev &v = views[find_view(tri_offs, nviews, g)];
                const int sh = __ffs(v.S) - 1;  // S is a power of two
                const int tx0 = (tb.x & 0xffff) >> sh, tx1 = (tb.x >> 16) >> sh;
                const int ty0 = (tb.y & 0xffff) >> sh;
                const int w = tx1 - tx0 + 1;
                const unsigned long long off = cand_off[e];
                const int q = (int)(p - (long long)off);  // < tiles of one view
                const int qy = q / w;
                const int tx = tx0 + (q - qy * w), ty = ty0 + qy;
                tile = v.tile_off + (long long)ty * v.tiles_x + tx;
                if (tx < 0 || ty < 0 || tx >= v.tiles_x || ty >= v.tiles_y) {  // never for a consistent bound
                    atomicOr(&cnt->status, ST_BAD_INDEX);
                    tile = v.tile_off;
                    ok_tile = false;
                }
                const float4 bb = rec[g * kRecF4 + 4];
                const bool fbspace = (tb.z & 0x100) != 0;
                const int nh = cand_off[e + 1] - off > 1 ? (tb.z & 0xff) : 0;
                if (!ok_tile) {
                    hit = false;
                } else if (!fbspace) {
                    hit = tile_meets(tile_box[tile], bb, hp + g * kMaxHp, nh);
                } else {
                    // the tile's pixel-centre box in framebuffer coordinates
                    const int i0 = tx << sh, i1 = min(v.W, (tx + 1) << sh) - 1;
                    const int j0 = ty << sh, j1 = min(v.H, (ty + 1) << sh) - 1;
                    const float4 fbt = make_float4(__fdiv_rn((float)i0 + 0.5f, (float)v.W),
                                                   __fdiv_rn((float)i1 + 0.5f, (float)v.W),
                                                   __fdiv_rn((float)j0 + 0.5f, (float)v.H),
                                                   __fdiv_rn((float)j1 + 0.5f, (float)v.H));
                    const float4 big = make_float4(-INFINITY, INFINITY, -INFINITY, INFINITY);
                    hit = tile_meets(tile_box[tile], bb, hp, 0) && tile_meets(fbt, big, hp + g * kMaxHp, nh);
                }
            }
            want_c[c] = __ballot_sync(0xffffffffu, hit);
            ent_c[c] = ((unsigned long long)key << 32) | (unsigned long long)g;
            tile_c[c] = (unsigned)tile;
        }
        // the task's hits go to the hit list with one atomic ...
        unsigned ntask = 0;
#pragma unroll
        for (int c = 0; c < kBinChunks; ++c)
            ntask += __popc(want_c[c]);
        if (ntask == 0)
            continue;
        unsigned long long wbase = 0;
        if (lane == 0)
            wbase = atomicAdd(&cnt->hits_listed, (unsigned long long)ntask);
        wbase = __shfl_sync(0xffffffffu, wbase, 0);
#pragma unroll
        for (int c = 0; c < kBinChunks; ++c) {
            const unsigned want = want_c[c];
            if (!want)
                continue;  // warp-uniform
            if ((want >> lane) & 1u) {
                const long long slot = (long long)wbase + __popc(want & ((1u << lane) - 1u));
                if (slot < cap_pairs) {
                    hit_entry[slot] = ent_c[c];
                    hit_tile[slot] = tile_c[c];
                } else {
                    atomicOr(&cnt->status, ST_OVERFLOW_PAIRS);
                }
                // ... and every tile's count with one atomic per tile met
                const unsigned peers = __match_any_sync(want, tile_c[c]);
                if (lane == __ffs(peers) - 1)
                    atomicAdd(&tile_cnt[tile_c[c]], (unsigned long long)__popc(peers));
            }
            wbase += __popc(want);
        }
    }
}

// Moves the listed hits into their tile bins (after the scan of the tile
// counts): entry k goes to scan[tile] + its rank among the tile's entries.
__global__ void __launch_bounds__(256) k_bin_scatter(const unsigned long long *__restrict__ hit_entry,
                                                     const unsigned *__restrict__ hit_tile,
                                                     const unsigned long long *__restrict__ scan,
                                                     unsigned int *__restrict__ fill,
                                                     unsigned long long *__restrict__ pairs, long long cap_pairs,
                                                     long long ntiles, Counters *cnt)
{
    const long long n = min((long long)cnt->hits_listed, cap_pairs);
    const int lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); k0 < n; k0 += stride) {
        const long long k = k0 + lane;
        bool ok = k < n;
        const unsigned tile = ok ? hit_tile[k] : 0u;
        if (ok && (long long)tile >= ntiles) {  // never for a consistent hit list
            atomicOr(&cnt->status, ST_BAD_INDEX);
            ok = false;
        }
        const unsigned want = __ballot_sync(0xffffffffu, ok);
        if (!ok)
            continue;
        // the bin start and the entry load while the cursor atomic runs
        const unsigned long long first = scan[tile] & 0xFFFFFFFFFFull;
        const unsigned long long ent = hit_entry[k];
        const unsigned peers = __match_any_sync(want, tile);
        const int leader = __ffs(peers) - 1;
        unsigned base = 0;
        if (lane == leader)
            base = atomicAdd(&fill[tile], (unsigned)__popc(peers));
        base = __shfl_sync(peers, base, leader);
        const long long pos = (long long)first + base + __popc(peers & ((1u << lane) - 1u));
        if (pos < cap_pairs)
            pairs[pos] = ent;
        else
            atomicOr(&cnt->status, ST_OVERFLOW_PAIRS);
    }
}

static int sm_count()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        n = sms > 0 ? sms : 1;
    }
    return n;
}

// k_bin_scatter: one wave of 256-thread CTAs (8 per SM)
static int bin_grid() { return sm_count() * 8; }

// k_bin: four waves of its four resident CTAs per SM (more waves measured
// the same, fewer slower; the binning stage of the 64-view workload took
// 0.43 ms with 2.7 waves of 3 CTAs per SM at 75 registers, 0.375 ms so)
static int bin_count_grid() { return sm_count() * 16; }

cudaError_t launch_bin_count(const ViewDev *views, int nviews, const long long *tri_offs, long long ttot,
                             const int *binned, const unsigned long long *cand_off, const float4 *rec,
                             const float4 *hp, const int4 *tbox, const float4 *tile_box, unsigned long long *tile_cnt,
                             unsigned long long *hit_entry, unsigned *hit_tile, long long cap_pairs, Counters *cnt,
                             cudaStream_t st)
{
    if (ttot > 0)
        k_bin<<<bin_count_grid(), 256, 0, st>>>(views, nviews, tri_offs, binned, cand_off, rec, hp, tbox,
                                                tile_box, tile_cnt, hit_entry, hit_tile, cap_pairs, cnt);
    return cudaGetLastError();
}

cudaError_t launch_bin_scatter(const unsigned long long *hit_entry, const unsigned *hit_tile,
                               const unsigned long long *scan, unsigned int *fill, unsigned long long *pairs,
                               long long cap_pairs, long long ntiles, Counters *cnt, cudaStream_t st)
{
    k_bin_scatter<<<bin_grid(), 256, 0, st>>>(hit_entry, hit_tile, scan, fill, pairs, cap_pairs, ntiles, cnt);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- frame init

// The start of a frame, in one launch: clears what the frame accumulates
// into -- the counters, the work-queue heads, the per-tile counts and fill
// cursors, the tickets and flags of two scans' look-back state
// (scan_state_words of each), the FP64 flag bitmap (nflag words, may be 0)
// -- sets every pixel's depth|id key to "no hit" (~0), and computes every
// tile's display box (stage a: the image of its pixel centres under q).
__global__ void k_frame_init(const ViewDev *__restrict__ views, int nviews, const long long *__restrict__ tile_offs,
                             float4 *__restrict__ tile_box, Counters *cnt, int *heads, unsigned long long *tile_cnt,
                             unsigned *fill, long long ntiles, unsigned long long *state_a, long long nstate_a,
                             unsigned long long *state_b, long long nstate_b, unsigned *flag_bits, long long nflag,
                             unsigned long long *keys, long long npix, float *loss_part, long long nloss)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    if (g == 0)
        *cnt = Counters{};
    if (g < 8)
        heads[g] = 0;
    for (long long k = g; k < ntiles; k += stride) {
        tile_cnt[k] = 0ull;
        fill[k] = 0u;
        tile_box[k] = tile_display_box(views, nviews, tile_offs, k);
    }
    for (long long k = g; k < nstate_a; k += stride)
        state_a[k] = 0ull;
    for (long long k = g; k < nstate_b; k += stride)
        state_b[k] = 0ull;
    for (long long k = g; k < nflag; k += stride)
        flag_bits[k] = 0u;
    for (long long k = g; k < nloss; k += stride)
        loss_part[k] = 0.f;
    // keys: 16-byte stores over the even-length prefix, then the last one
    ulonglong2 *k2 = reinterpret_cast<ulonglong2 *>(keys);
    for (long long k = g; k < npix / 2; k += stride)
        k2[k] = make_ulonglong2(~0ull, ~0ull);
    if (g == 0 && (npix & 1))
        keys[npix - 1] = ~0ull;
}

cudaError_t launch_frame_init(const ViewDev *views, int nviews, const long long *tile_offs, float4 *tile_box,
                              Counters *cnt, int *heads, unsigned long long *tile_cnt, unsigned *fill, long long ntiles,
                              unsigned long long *state_a, long long nstate_a, unsigned long long *state_b,
                              long long nstate_b, unsigned *flag_bits, long long nflag, unsigned long long *keys,
                              long long npix, float *loss_part, long long nloss, cudaStream_t st)
{
    static int grid = 0;
    if (grid == 0) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        grid = sms * 8;
    }
    k_frame_init<<<grid, 256, 0, st>>>(views, nviews, tile_offs, tile_box, cnt, heads, tile_cnt, fill, ntiles, state_a,
                                       nstate_a, state_b, nstate_b, flag_bits, nflag, keys, npix, loss_part, nloss);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- scan

// Exclusive prefix sum of u64 words in one pass (decoupled look-back,
// Merrill and Garland 2016): each CTA scans a tile of kScanBlock words,
// publishes the tile's sum, and warp 0 walks back over its predecessors --
// 32 at a time, polling their flags -- until it meets a tile whose
// inclusive prefix is published.  Tiles are numbered by an atomic ticket,
// so every tile waited on belongs to a CTA that started earlier; each poll
// is bounded (ST_TIMEOUT if it runs out).  With seg > 0 each input word is
// first packed as low 40 bits = bin entries, high 24 bits = work items
// (ceil(entries / seg)).  out[n] = the grand total.
constexpr int kScanThreads = 512, kScanPer = 8, kScanBlock = kScanThreads * kScanPer;
constexpr unsigned long long kFlagAgg = 1ull, kFlagPre = 2ull;
constexpr int kScanSpinLimit = 1 << 22;

__device__ __forceinline__ unsigned long long pack_items(unsigned long long c, int seg)
{
    const unsigned long long n = c & 0xFFFFFFFFFFull;
    // a 32-bit division where the count allows it (a 64-bit one is a long
    // instruction sequence)
    const unsigned long long items = n <= 0x7FFFFFFFull
                                         ? (unsigned long long)(((unsigned)n + (unsigned)seg - 1u) / (unsigned)seg)
                                         : (n + seg - 1) / seg;
    return n | (items << 40);
}

__device__ unsigned long long block_exclusive_scan(unsigned long long x, unsigned long long *total)
{
    __shared__ unsigned long long warp_sums[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long inc = x;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o)
            inc += y;
    }
    if (lane == 31)
        warp_sums[w] = inc;
    __syncthreads();
    if (w == 0) {
        unsigned long long s = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0ull;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o)
                s += y;
        }
        warp_sums[lane] = s;
    }
    __syncthreads();
    const unsigned long long before = w > 0 ? warp_sums[w - 1] : 0ull;
    *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + inc - x;
}

__device__ __forceinline__ unsigned long long load_volatile(const unsigned long long *p)
{
    return *(const volatile unsigned long long *)p;
}
__device__ __forceinline__ void store_volatile(unsigned long long *p, unsigned long long v)
{
    *(volatile unsigned long long *)p = v;
}

// state: [0] ticket, [1, 1 + nb) flags, then nb tile sums, then nb
// inclusive prefixes; the ticket and flags start at zero.  gather: element
// i is in[gather[i]] (else in[i]).  n_dev: the element count is
// min(*n_dev, n), known on the device only; tiles past it leave at once.
// Emits the work items of tile g from its bin count n and its exclusive
// prefix (bin entries, low 40 bits; work items, high 24): the bin cut into
// runs of at most seg triangles, item = (view, tile in view, first entry,
// end entry).  Runs past the bin buffer (its scatter overflowed) are clamped
// to it, so the frame stays in bounds; the overflow status reruns it.
__device__ __forceinline__ void emit_items(const ItemsOut &io, long long g, long long n, unsigned long long pre,
                                           int seg, Counters *cnt)
{
    if (n == 0)
        return;
    const int vi = find_view(io.tile_offs, io.nviews, g);
    const long long lt = g - io.views[vi].tile_off;
    const long long off = (long long)(pre & 0xFFFFFFFFFFull), ioff = (long long)(pre >> 40);
    const long long nit = (n + seg - 1) / seg;
    for (long long q = 0; q < nit; ++q) {
        const long long b0 = min(off + q * seg, io.cap_pairs), b1 = min(off + min(n, (q + 1) * seg), io.cap_pairs);
        if (ioff + q < io.cap_items)
            io.items[ioff + q] = make_int4(vi, (int)lt, (int)b0, (int)b1);
        else
            atomicOr(&cnt->status, ST_OVERFLOW_ITEMS);
    }
}

template <bool kItems>
__global__ void __launch_bounds__(kScanThreads) k_scan(const unsigned long long *__restrict__ in,
                                                      const int *__restrict__ gather,
                                                      const unsigned long long *__restrict__ n_dev,
                                                      unsigned long long *__restrict__ out, long long n, int seg,
                                                      unsigned long long *state, long long nb, Counters *cnt,
                                                      ItemsOut io, int spin_limit)
{
    unsigned long long *flags = state + 1, *agg = state + 1 + nb, *inc = state + 1 + 2 * nb;
    __shared__ long long s_tile;
    __shared__ unsigned long long s_excl;
    if (threadIdx.x == 0)
        s_tile = (long long)atomicAdd(&state[0], 1ull);
    __syncthreads();
    const long long tile = s_tile;
    if (n_dev) {
        n = min(n, (long long)*n_dev);
        // tiles are numbered in start order, so no tile at or before the
        // one that holds out[n] waits on these
        if (tile * kScanBlock > n)
            return;
    }
    const long long base = tile * kScanBlock + (long long)threadIdx.x * kScanPer;
    unsigned long long v[kScanPer], sum = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        unsigned long long x = 0ull;
        if (base + k < n)
            x = in[gather ? (long long)gather[base + k] : base + k];
        v[k] = seg > 0 ? pack_items(x, seg) : x;
        sum += v[k];
    }
    unsigned long long total;
    unsigned long long run = block_exclusive_scan(sum, &total);
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        unsigned long long excl = 0;
        if (tile == 0) {
            if (lane == 0) {
                store_volatile(&inc[0], total);
                __threadfence();
                store_volatile(&flags[0], kFlagPre);
            }
        } else {
            if (lane == 0) {
                store_volatile(&agg[tile], total);
                __threadfence();
                store_volatile(&flags[tile], kFlagAgg);
            }
            bool late = false;
            for (long long j = tile - 1;; j -= 32) {
                const long long t = j - lane;
                unsigned long long f = kFlagPre, val = 0;  // before tile 0: a prefix of 0
                if (t >= 0) {
                    int spins = 0;
                    while ((f = load_volatile(&flags[t])) == 0ull) {
                        if (++spins > spin_limit) {
                            late = true;
                            f = kFlagPre;
                            break;
                        }
                        __nanosleep(32);
                    }
                    __threadfence();
                    if (f == kFlagPre)
                        val = load_volatile(&inc[t]);
                    else
                        val = load_volatile(&agg[t]);
                }
                const unsigned pre = __ballot_sync(0xffffffffu, f == kFlagPre);
                const int first = pre ? __ffs(pre) - 1 : 31;  // nearest tile with a prefix
                unsigned long long c = lane <= first ? val : 0ull;
                for (int o = 16; o > 0; o >>= 1)
                    c += __shfl_xor_sync(0xffffffffu, c, o);
                excl += c;
                if (pre)
                    break;
            }
            if (lane == 0) {
                store_volatile(&inc[tile], excl + total);
                __threadfence();
                store_volatile(&flags[tile], kFlagPre);
            }
            if (__any_sync(0xffffffffu, late) && lane == 0)
                atomicOr(&cnt->status, ST_TIMEOUT);
        }
        if (lane == 0)
            s_excl = excl;
    }
    __syncthreads();
    const unsigned long long excl = s_excl;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        if (base + k < n) {
            out[base + k] = excl + run;
            if (kItems)
                emit_items(io, base + k, (long long)(v[k] & 0xFFFFFFFFFFull), excl + run, seg, cnt);
        }
        run += v[k];
    }
    const bool holds_end =
        (n >= tile * kScanBlock && n < (tile + 1) * kScanBlock) || (tile == nb - 1 && n == nb * kScanBlock);
    if (threadIdx.x == 0 && holds_end) {
        out[n] = excl + total;
        if (kItems) {
            cnt->pairs_total = (excl + total) & 0xFFFFFFFFFFull;
            cnt->items_total = (excl + total) >> 40;
        }
    }
}

long long scan_state_words(long long n)
{
    return (n + kScanBlock - 1) / kScanBlock + 1;
}

size_t scan_block_sums_needed(long long n)
{
    const long long nb = (n + kScanBlock - 1) / kScanBlock;
    return (size_t)(3 * nb + 2);
}

cudaError_t launch_scan(const unsigned long long *in, unsigned long long *out, unsigned long long *state, long long n,
                        int seg, Counters *cnt, cudaStream_t st, bool state_zeroed, const int *gather,
                        const unsigned long long *n_dev, const ItemsOut *items)
{
    const long long nb = (n + kScanBlock - 1) / kScanBlock;
    if (nb == 0) {
        cudaMemsetAsync(out, 0, sizeof(unsigned long long), st);
        return cudaGetLastError();
    }
    if (!state_zeroed) {
        cudaError_t e = cudaMemsetAsync(state, 0, sizeof(unsigned long long) * (nb + 1), st);
        if (e != cudaSuccess)
            return e;
    }
    if (items && seg > 0)
        k_scan<true><<<(unsigned)nb, kScanThreads, 0, st>>>(in, gather, n_dev, out, n, seg, state, nb, cnt, *items,
                                                            kScanSpinLimit);
    else
        k_scan<false><<<(unsigned)nb, kScanThreads, 0, st>>>(in, gather, n_dev, out, n, seg, state, nb, cnt,
                                                             ItemsOut{}, kScanSpinLimit);
    return cudaGetLastError();
}

// Failure detection of the look-back wait, without a fault: a two-tile scan
// launched as ONE block whose ticket is preset to 1, so its predecessor
// (tile 0) never runs and never publishes.  The block polls tile 0's flag
// until the (here short) spin limit runs out, sets ST_TIMEOUT and finishes;
// every access stays inside the buffers.  Returns the status word.
cudaError_t scan_timeout_probe(cudaStream_t st, unsigned *status)
{
    const long long n = 2 * kScanBlock, nb = 2;
    unsigned long long *in = nullptr, *out = nullptr, *state = nullptr;
    Counters *cnt = nullptr;
    *status = 0u;
    cudaError_t e = cudaMalloc(&in, sizeof(unsigned long long) * n);
    if (e == cudaSuccess)
        e = cudaMalloc(&out, sizeof(unsigned long long) * (n + 1));
    if (e == cudaSuccess)
        e = cudaMalloc(&state, sizeof(unsigned long long) * scan_block_sums_needed(n));
    if (e == cudaSuccess)
        e = cudaMalloc(&cnt, sizeof(Counters));
    if (e == cudaSuccess)
        e = cudaMemsetAsync(in, 0, sizeof(unsigned long long) * n, st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(state, 0, sizeof(unsigned long long) * scan_block_sums_needed(n), st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(cnt, 0, sizeof(Counters), st);
    if (e == cudaSuccess) {
        const unsigned long long one = 1ull;  // the ticket: the only block becomes tile 1
        e = cudaMemcpyAsync(state, &one, sizeof one, cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) {
        k_scan<false><<<1, kScanThreads, 0, st>>>(in, nullptr, nullptr, out, n, 0, state, nb, cnt, ItemsOut{},
                                                  1 << 12);
        e = cudaGetLastError();
    }
    Counters h{};
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&h, cnt, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e == cudaSuccess)
        *status = h.status;
    cudaFree(in);
    cudaFree(out);
    cudaFree(state);
    cudaFree(cnt);
    return e;
}

// ---------------------------------------------------------------- run sort

// Sorts the bin run of every work item by depth key, nearest first, so the
// fragment stage can stop a run at the first triangle that lies behind
// every pixel of its block.  One warp per item.  A run of up to 256 entries
// is sorted in registers (R = 1, 2, 4 or 8 per lane) by a bitonic network
// over 32-bit words: the depth order key with its low 8 bits replaced by
// the entry's position in the run.  The entry is written back with that
// truncated key -- a lower bound of the true one, so every cut the fragment
// stage takes on it stays conservative -- and its triangle index.  Longer
// runs (pr_params.seg above 256) are sorted in the warp's shared memory on
// the full 64-bit entries.
constexpr int kSortWarps = 4;
constexpr int kSortRegMax = 256;

template <int R>
__device__ __forceinline__ void warp_bitonic(unsigned (&x)[R], int lane)
{
    // element m of a lane sits at position 32 m + lane
#pragma unroll
    for (int k = 2; k <= 32 * R; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
#pragma unroll
                for (int m = 0; m < R; ++m) {
                    const int m2 = m ^ (j >> 5);
                    if (m2 > m) {
                        const bool up = ((32 * m) & k) == 0;
                        const unsigned lo = min(x[m], x[m2]), hi = max(x[m], x[m2]);
                        x[m] = up ? lo : hi;
                        x[m2] = up ? hi : lo;
                    }
                }
            } else {
#pragma unroll
                for (int m = 0; m < R; ++m) {
                    const unsigned y = __shfl_xor_sync(0xffffffffu, x[m], j);
                    // the lower position of a pair keeps the smaller word in
                    // an ascending block, the larger in a descending one
                    const bool lower = (lane & j) == 0, up = ((32 * m + lane) & k) == 0;
                    x[m] = (lower == up) ? min(x[m], y) : max(x[m], y);
                }
            }
        }
    }
}

template <int R>
__device__ __forceinline__ void sort_run_regs(unsigned long long *e, int n, int lane, unsigned *s_gid)
{
    unsigned x[R];
#pragma unroll
    for (int m = 0; m < R; ++m) {
        const int q = 32 * m + lane;
        if (q < n) {
            const unsigned long long v = e[q];
            x[m] = ((unsigned)(v >> 32) & ~0xFFu) | (unsigned)q;
            s_gid[q] = (unsigned)v;
        } else {
            x[m] = 0xFFFFFFFFu;  // above every real word (keys are finite or +-inf)
        }
    }
    __syncwarp();
    warp_bitonic<R>(x, lane);
#pragma unroll
    for (int m = 0; m < R; ++m) {
        const int q = 32 * m + lane;
        if (q < n)
            e[q] = ((unsigned long long)(x[m] & ~0xFFu) << 32) | s_gid[x[m] & 0xFFu];
    }
    __syncwarp();
}

template <bool kLong>
__global__ void __launch_bounds__(kSortWarps * 32) k_sort_items(const int4 *__restrict__ items,
                                                                const unsigned long long *__restrict__ scan,
                                                                long long ntiles, long long cap_items,
                                                                unsigned long long *__restrict__ pairs,
                                                                const Counters *__restrict__ cnt)
{
    if (cnt->status & (ST_OVERFLOW_PAIRS | ST_OVERFLOW_ITEMS | ST_TIMEOUT))
        return;  // an overflowed attempt (rerun) or a scan that gave up its wait (an error): bins incomplete
    __shared__ unsigned s_gid[kSortWarps][kSortRegMax];
    __shared__ unsigned long long s_run[kSortWarps][kLong ? kMaxSeg : 1];
    const long long nitems = min((long long)(scan[ntiles] >> 40), cap_items);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long *run = s_run[w];
    const long long nwarps = (long long)gridDim.x * kSortWarps;
    for (long long it = (long long)blockIdx.x * kSortWarps + w; it < nitems; it += nwarps) {
        const int4 item = items[it];
        const int n = item.w - item.z;
        unsigned long long *e = pairs + item.z;
        if (n <= 1)
            continue;
        if (n <= 32) {
            sort_run_regs<1>(e, n, lane, s_gid[w]);
            continue;
        }
        if (n <= 64) {
            sort_run_regs<2>(e, n, lane, s_gid[w]);
            continue;
        }
        if (n <= 128) {
            sort_run_regs<4>(e, n, lane, s_gid[w]);
            continue;
        }
        if (n <= kSortRegMax || !kLong) {  // without kLong, runs are at most kSortRegMax long
            sort_run_regs<8>(e, n, lane, s_gid[w]);
            continue;
        }
        int P = 512;
        while (P < n)
            P <<= 1;
        for (int q = lane; q < P; q += 32)
            run[q] = q < n ? e[q] : ~0ull;
        __syncwarp();
        for (int k = 2; k <= P; k <<= 1)
            for (int j = k >> 1; j > 0; j >>= 1) {
                for (int q = lane; q < P / 2; q += 32) {
                    // q-th compare-exchange pair of this step: (i, i + j)
                    const int i = ((q & ~(j - 1)) << 1) | (q & (j - 1));
                    const unsigned long long a = run[i], b = run[i + j];
                    const bool up = (i & k) == 0;
                    if ((a > b) == up) {
                        run[i] = b;
                        run[i + j] = a;
                    }
                }
                __syncwarp();
            }
        for (int q = lane; q < n; q += 32)
            e[q] = run[q];
        __syncwarp();
    }
}

cudaError_t launch_sort_items(const int4 *items, const unsigned long long *scan, long long ntiles, long long cap_items,
                              int seg, unsigned long long *pairs, const Counters *cnt, cudaStream_t st)
{
    // 32 CTAs of four warps per SM, about three waves: the warps take the
    // items grid-stride, and runs of very different lengths even out when
    // late CTAs fill the slots of early ones (the 64-view workload's binning
    // stage 0.371 -> 0.365 ms against 8 CTAs per SM)
    const int grid = sm_count() * 32;
    if (seg > kSortRegMax)
        k_sort_items<true><<<grid, kSortWarps * 32, 0, st>>>(items, scan, ntiles, cap_items, pairs, cnt);
    else
        k_sort_items<false><<<grid, kSortWarps * 32, 0, st>>>(items, scan, ntiles, cap_items, pairs, cnt);
    return cudaGetLastError();
}

}  // namespace pr
