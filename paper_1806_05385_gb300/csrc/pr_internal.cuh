// pr_internal.cuh -- device-side records and math shared by the kernels of
// libpr (stages (a)-(e) of the perceptual-rasterization hot path).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "../../include/pr.h"

namespace pr {

constexpr float kSqrt2 = 1.41421356237309504880f;  // D, the extent of the foveation domain (Sec. 3.1.1)
constexpr float kEpsDisp = 1e-5f;                  // display-space safety margin of every bound (unit coords)
constexpr float kEpsT = 1e-4f;                     // time margin of every catch-up interval
constexpr int kMaxHp = 8;                          // half-planes per bound: <= 6 hull edges + 2 time-strip edges
constexpr int kRecF4 = 6;                          // float4 per fragment record
// the pixel block of one warp in shading and the adjoint (32 pixels)
constexpr int kBlkW = 8, kBlkH = 4;
static_assert(kBlkW * kBlkH == 32, "one pixel per lane");
__host__ __device__ inline long long pixel_blocks(int W, int H)
{
    return (long long)((W + kBlkW - 1) / kBlkW) * ((H + kBlkH - 1) / kBlkH);
}
constexpr int kMaxSeg = 1024;                      // longest bin run of one work item (pr_params.seg)
constexpr int kLossSlots = 256;                    // partial sums per view of a training frame's loss

// Device status bits (Counters::status).
enum : uint32_t {
    ST_OVERFLOW_PAIRS = 1u,
    ST_OVERFLOW_ITEMS = 2u,
    ST_TIMEOUT = 4u,
    ST_NONFINITE = 8u,
    ST_BAD_INDEX = 16u,
    ST_OVERFLOW_FLAGS = 32u,
};

// Per-view constants, derived on the host from pr_view (see pr_host.cu).
struct ViewDev {
    float R0[9], T0[3], R1[9], T1[3];  // pose0 / pose1 as rotation + translation
    float tan_x, tan_y, z_near;
    float fx, fy;                      // fovea x_f (unit framebuffer coordinates)
    float alpha, inv_alpha;            // p(d) = D (d/D)^alpha (when p_lut is null)
    const float *p_lut;                // or: p sampled at d_k = k D / p_n (device)
    int p_n;
    float d0, d1;                      // rolling direction, r(x) = x . d
    float t_lo, t_hi;                  // range of pixel times over the viewport
    float l0[3], l1[3];                // camera-space light direction at t = 0 and t = 1
    float k_a, k_d, k_s, shininess;
    int W, H, mode, S;                 // framebuffer, pr_mode, bin tile side
    int tiles_x, tiles_y, bound, fp64;
    int fov_bound;                     // pr_fov_bound
    long long tri_off, tile_off, pix_off;  // offsets of this view in the batch-wide arrays
    long long blk_off;                 // offset of its warp pixel blocks (stages d, e)
    int T, V;
    const float4 *vtx;                 // scene vertices, two float4 each: (px, py, pz, vx), (vy, vz, 0, 0)
    const float4 *col4;                // per-vertex colour (r, g, b, 0)
    const int4 *tri4;                  // per-triangle vertex indices (i0, i1, i2, 0)
    uint32_t *id_out;                  // resolved outputs (device)
    float *depth_out;
    const uint32_t *id_in;             // ids read by shading / adjoint
    float *rgb_out;
    const float *grad_in;              // adjoint input [3][H][W]
    const float *target;               // or: L2 target [3][H][W], gradient 2 (rgb - target) from rgb_out
    const unsigned char *target_u8;    // or: 8-bit L2 target [3][H][W] (value / 255)
    float *loss;                       // L2 loss of the view, accumulated (+=), or null
    float *loss_part;                  // kLossSlots partial sums of it (workspace; cleared by the frame init)
    const unsigned *scene_status;      // the scene's status word (ST_NONFINITE after an update), or null
    float *dcol, *dpos, *dvel;         // adjoint outputs [V][3]
    const float4 *rec;                 // this frame's stage (a) records (batch-wide index), or null
    unsigned long long bw_mul;         // ceil(2^40 / bw), bw = 8-pixel blocks per row: lb / bw = (lb * bw_mul) >> 40
};

// The views of a launch passed by value in the kernel's parameter space, for
// batches of up to kParamViews views (72 x 416 bytes, within the 32 KB a
// launch may pass).  A kernel then reads their fields through the constant
// cache (warp-uniform, off the L1 path) and can re-read one instead of
// holding it in a register.  Larger batches read the device table.
constexpr int kParamViews = 72;
struct ParamViews {
    ViewDev v[kParamViews];
};
static_assert(sizeof(ParamViews) <= 30 * 1024, "the view table must fit the kernel parameter space");

struct Counters {
    unsigned long long tests, hits, culled, flagged, changed;
    unsigned long long pairs_total, items_total;  // copied from the scan for the host
    unsigned long long hits_listed;               // (triangle, tile) hits appended by the binning count pass
    unsigned long long binned;                    // triangles with candidate tiles, listed by the bound pass
    unsigned int status;
    unsigned int depth_err_bits;  // bits of the largest FP32-vs-FP64 relative depth error (re-test)
};

__device__ __forceinline__ bool is_rolling(int mode) { return mode == PR_ROLLING || mode == PR_BOTH; }
__device__ __forceinline__ bool is_foveated(int mode) { return mode == PR_FOVEATED || mode == PR_BOTH; }

// Index of the view that owns element g, given the batch offsets off[0..n]
// (off[0] = 0, ascending).
__device__ __forceinline__ int find_view(const long long *off, int n, long long g)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= g)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// The same for a g that every lane of the warp holds: the lanes compare 32
// offsets at a time (one load each, no chain of dependent loads) and count
// those at or below g.  Called by the whole warp.
__device__ __forceinline__ int find_view_warp(const long long *off, int n, long long g)
{
    const int lane = threadIdx.x & 31;
    int q = 0;
    for (int base = 1; base < n; base += 32) {
        const int k = base + lane;
        const unsigned m = __ballot_sync(0xffffffffu, k < n && off[k] <= g);
        q += __popc(m);
        if (m != 0xffffffffu)
            break;  // offsets ascend: none further on is at or below g
    }
    return q;
}

// Camera-space start and end positions of vertex k: S = R0 p + T0 and
// E = R1 (p + v) + T1 (Sec. 3.2, "Bounding": M_s v_s and M_e v_e).  Every
// kernel that needs a vertex calls this one function, so the bits agree.
__device__ __forceinline__ void vertex_start_end(const ViewDev &v, int k, float3 &S, float3 &E)
{
    const float4 a = v.vtx[2 * k], b = v.vtx[2 * k + 1];  // one 32-byte sector
    const float x = a.x, y = a.y, z = a.z;
    const float ex = x + a.w, ey = y + b.x, ez = z + b.y;
    S.x = fmaf(v.R0[0], x, fmaf(v.R0[1], y, fmaf(v.R0[2], z, v.T0[0])));
    S.y = fmaf(v.R0[3], x, fmaf(v.R0[4], y, fmaf(v.R0[5], z, v.T0[1])));
    S.z = fmaf(v.R0[6], x, fmaf(v.R0[7], y, fmaf(v.R0[8], z, v.T0[2])));
    E.x = fmaf(v.R1[0], ex, fmaf(v.R1[1], ey, fmaf(v.R1[2], ez, v.T1[0])));
    E.y = fmaf(v.R1[3], ex, fmaf(v.R1[4], ey, fmaf(v.R1[5], ez, v.T1[1])));
    E.z = fmaf(v.R1[6], ex, fmaf(v.R1[7], ey, fmaf(v.R1[8], ez, v.T1[2])));
}

// A foveation function given by samples (Sec. 3.1.1, any monotonic p): p
// linear between p_k = p(k D / n) (the last segment continued), p^-1 its
// exact inverse.  Used by every stage when a view has samples.
struct SampledP {
    const float *lut;
    int n;
    __host__ __device__ float p(float d) const
    {
        const float x = d * ((float)n / kSqrt2);
        int k = (int)floorf(x);
        k = k < 0 ? 0 : (k > n - 1 ? n - 1 : k);
        const float t = x - (float)k;
        return fmaf(t, lut[k + 1] - lut[k], lut[k]);
    }
    __host__ __device__ int segment(float r) const  // last k with lut[k] <= r
    {
        int lo = 0, hi = n - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (lut[mid] <= r)
                lo = mid;
            else
                hi = mid - 1;
        }
        return lo;
    }
    __host__ __device__ float pinv(float r) const
    {
        const int k = segment(r);
        return ((float)k + (r - lut[k]) / (lut[k + 1] - lut[k])) * (kSqrt2 / (float)n);
    }
    __host__ __device__ float dpinv(float r) const  // slope of p^-1 at r
    {
        const int k = segment(r);
        return (kSqrt2 / (float)n) / (lut[k + 1] - lut[k]);
    }
};

// Foveation q (framebuffer -> display) of a point at offset e from the
// fovea: the offset is scaled by p(|e|)/|e| = (|e|/D)^(alpha-1).
__device__ __forceinline__ float fov_scale(float r, float alpha)
{
    return r > 0.f ? __powf(r * (1.0f / kSqrt2), alpha - 1.0f) : 0.f;
}

// Pixel (i, j) -> its display location x, its time t and its ray direction
// (dx, dy, 1) (conventions of pr.h).  FP32; the same code in every stage.
// kLut = false: the caller knows no view uses a sampled p, and the sampled
// path is left out (same results for the power map, fewer registers).
template <bool kLut = true>
__device__ __forceinline__ void pixel_ray(const ViewDev &v, int i, int j, float &x0, float &x1, float &t, float &dx,
                                          float &dy)
{
    float u0 = __fdiv_rn((float)i + 0.5f, (float)v.W);
    float u1 = __fdiv_rn((float)j + 0.5f, (float)v.H);
    if (is_foveated(v.mode)) {
        float e0 = u0 - v.fx, e1 = u1 - v.fy;
        float r = sqrtf(fmaf(e0, e0, e1 * e1));
        float s;
        if (kLut && v.p_lut) {  // sampled p: the offset scaled by p(r) / r (the first slope at r = 0)
            const SampledP sp{v.p_lut, v.p_n};
            s = r > 0.f ? sp.p(r) / r : sp.lut[1] * ((float)sp.n / kSqrt2);
        } else {
            s = fov_scale(r, v.alpha);
        }
        x0 = fmaf(e0, s, v.fx);
        x1 = fmaf(e1, s, v.fy);
    } else {
        x0 = u0;
        x1 = u1;
    }
    t = is_rolling(v.mode) ? fmaf(x0, v.d0, x1 * v.d1) : 0.f;
    dx = fmaf(2.f, x0, -1.f) * v.tan_x;
    dy = fmaf(2.f, x1, -1.f) * v.tan_y;
}

// The pixel's time and ray in FP64 from the same inputs (the FP32 view
// constants widen exactly): u = ((i + 1/2)/W, (j + 1/2)/H), x = q(u) when
// foveated, t = x . d when rolling, dir = ((2 x0 - 1) tanX, (2 x1 - 1) tanY, 1).
struct Ray64 {
    double t, dx, dy;
};

__device__ inline Ray64 pixel_ray64(const ViewDev &v, int i, int j)
{
    double x0 = ((double)i + 0.5) / (double)v.W, x1 = ((double)j + 0.5) / (double)v.H;
    if (is_foveated(v.mode)) {
        const double f0 = v.fx, f1 = v.fy;
        const double e0 = x0 - f0, e1 = x1 - f1;
        const double r = sqrt(e0 * e0 + e1 * e1);
        if (r > 0.0) {
            double s;
            if (v.p_lut) {  // the sampled p, linear between the samples, in FP64
                const double D = 1.4142135623730950488, xk = r * (double)v.p_n / D;
                int k = (int)floor(xk);
                k = k < 0 ? 0 : (k > v.p_n - 1 ? v.p_n - 1 : k);
                const double t = xk - (double)k;
                s = ((1.0 - t) * (double)v.p_lut[k] + t * (double)v.p_lut[k + 1]) / r;
            } else {
                // (r / D)^(alpha - 1); the integer exponents of the usual
                // power maps exactly or by one rounded product
                const double xr = r / 1.4142135623730950488;
                s = v.alpha == 2.f ? xr : (v.alpha == 3.f ? xr * xr : pow(xr, (double)v.alpha - 1.0));
            }
            x0 = f0 + e0 * s;
            x1 = f1 + e1 * s;
        } else {
            x0 = f0;
            x1 = f1;
        }
    }
    Ray64 ry;
    ry.t = is_rolling(v.mode) ? x0 * (double)v.d0 + x1 * (double)v.d1 : 0.0;
    ry.dx = (2.0 * x0 - 1.0) * (double)v.tan_x;
    ry.dy = (2.0 * x1 - 1.0) * (double)v.tan_y;
    return ry;
}

// Display location (unit coordinates) of a camera-space point with z > 0.
__device__ __forceinline__ float2 project(const ViewDev &v, float3 p)
{
    float iz = 1.0f / p.z;
    return make_float2(fmaf(0.5f * p.x * iz, 1.0f / v.tan_x, 0.5f), fmaf(0.5f * p.y * iz, 1.0f / v.tan_y, 0.5f));
}

// A float as an unsigned integer of the same order (negative values
// included), and back: the depth sort key of the bin pairs.
__host__ __device__ __forceinline__ uint32_t depth_order_key(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    return u ^ ((u >> 31) ? 0xFFFFFFFFu : 0x80000000u);
}
__host__ __device__ __forceinline__ float depth_from_order_key(uint32_t u)
{
    u ^= (u >> 31) ? 0x80000000u : 0xFFFFFFFFu;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

// Packed visibility key: FP32 depth bits (positive floats order as their
// bits) above the triangle id, so a 64-bit min picks the nearest hit and,
// on equal depth, the smaller id.
__device__ __forceinline__ unsigned long long pack_key(float depth, uint32_t id)
{
    return ((unsigned long long)__float_as_uint(depth) << 32) | (unsigned long long)id;
}

}  // namespace pr
