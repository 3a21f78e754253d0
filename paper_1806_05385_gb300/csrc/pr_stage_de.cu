// pr_stage_de.cu -- stage (d): deferred shading at the pixel time (Sec. 3.2,
// "Shading"), and stage (e): its adjoint with respect to the vertex colours,
// positions and velocities, with the visible triangle of every pixel held
// fixed.  Both recompute the pixel's time, ray, moved triangle and
// barycentrics from the id buffer instead of storing them.
#include "pr_launch.h"

#include <cstring>

namespace pr {

__device__ __forceinline__ float3 sub3(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ float3 cross3(float3 a, float3 b)
{
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
// The same cross product with every rounding fixed (no contraction left to
// the compiler), so that every kernel that shades a pixel gets the same bits.
__device__ __forceinline__ float3 cross3_rn(float3 a, float3 b)
{
    return make_float3(fmaf(a.y, b.z, -__fmul_rn(a.z, b.y)), fmaf(a.z, b.x, -__fmul_rn(a.x, b.z)),
                       fmaf(a.x, b.y, -__fmul_rn(a.y, b.x)));
}
__device__ __forceinline__ float3 scale3(float3 a, float s) { return make_float3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float3 add3(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }

// An 8-bit value b as b / 255 without the conversion pipe: 2^23 + b is exact
// in FP32 (its bits are 0x4B000000 | b), so subtracting 2^23 leaves b
// exactly; the product is the correctly rounded b * (1/255 in FP32), the
// same as (float)b * (1.f / 255.f).
__device__ __forceinline__ float u8_unit(unsigned char b)
{
    return (__uint_as_float(0x4B000000u | (unsigned)b) - 8388608.f) * (1.f / 255.f);
}

// Everything shading needs about the visible triangle at one pixel.
struct PixelHit {
    int ia, ib, ic;     // vertex indices
    float t;            // pixel time
    float3 dir;         // ray direction
    float3 A, B, C;     // triangle moved to t (camera space)
    float b0, b1, b2;   // barycentrics of the ray point
    float det;          // U + V + W of the watertight test
    float inv_det;      // 1 / det (0 if det = 0)
    float3 n;           // unit normal facing the viewer
    float inl;          // flip / |(B-A) x (C-A)| with flip = +-1 the sign applied (0 if degenerate)
    float3 l;           // unit light direction at t
    float ndl, sigma;   // n.l and k_a + k_d max(0, n.l)
    float3 hv;          // Blinn-Phong half vector normalize(l + v), v = the reversed ray
    float ndh, spec;    // n.h and k_s max(0, n.h)^shininess (0 without specular)
};

// Paths the shading kernels are built with: a view of the launch may have a
// specular term (k_s > 0), a view may use a sampled foveation function, a
// view may ask for the precision form.  The kernels built without a path
// are faster (fewer registers); the results of the views they shade are the
// same bits.
constexpr int kFeatSpec = 1, kFeatLut = 2, kFeatF64 = 4;

// Precision form of the shading: the FP32 barycentrics of a triangle that
// is small against its distance carry an error of about (coordinate error)
// x (sheared extent) / |det|, that is one coordinate ulp over the
// triangle's size; a pixel whose estimate exceeds kBaryRel takes its moved
// triangle, barycentrics and normal from FP64 instead (the FP32 coordinate
// error is taken as kRelCoordShade of the magnitudes it came from, about
// one ulp: measured colour errors of such triangles match it).
constexpr float kBaryRel = 2e-5f;
constexpr float kRelCoordShade = 6e-8f;

// The pixel's moved triangle, barycentrics and unit normal in FP64 from the
// scene's FP32 inputs (widened exactly), rounded to FP32 into h: the
// interpolation of M_s v_s and M_e v_e at the pixel time, the ray-plane
// barycentrics b_k = w_k / sum w with w_0 = dir.(B x C) (cyclically) and the
// face normal turned to face the viewer.
__device__ __noinline__ void pixel_hit64(const ViewDev &v, int i, int j, struct PixelHit &h);

template <int kFeat>
__device__ __forceinline__ void pixel_hit(const ViewDev &v, int i, int j, unsigned id, PixelHit &h)
{
    float x0, x1, dx, dy;
    pixel_ray<(kFeat & kFeatLut) != 0>(v, i, j, x0, x1, h.t, dx, dy);
    h.dir = make_float3(dx, dy, 1.f);
    const int4 tv = v.tri4[id];
    h.ia = tv.x;
    h.ib = tv.y;
    h.ic = tv.z;
    const float t = h.t;
    if (v.rec) {
        // the frame's own stage (a) record: S and D = E - S, the same bits
        // vertex_start_end gives, in 64 contiguous bytes
        const float4 *r = v.rec + ((size_t)v.tri_off + id) * kRecF4;
        const float4 r0 = r[0], r1 = r[1], r2 = r[2], r3 = r[3], r5 = r[5];
        h.A = make_float3(fmaf(t, r2.y, r0.x), fmaf(t, r2.z, r0.y), fmaf(t, r2.w, r0.z));
        h.B = make_float3(fmaf(t, r3.x, r0.w), fmaf(t, r3.y, r1.x), fmaf(t, r3.z, r1.y));
        h.C = make_float3(fmaf(t, r3.w, r1.z), fmaf(t, r5.z, r1.w), fmaf(t, r5.w, r2.x));
    } else {
        float3 S, E;
        vertex_start_end(v, h.ia, S, E);
        h.A = make_float3(fmaf(t, E.x - S.x, S.x), fmaf(t, E.y - S.y, S.y), fmaf(t, E.z - S.z, S.z));
        vertex_start_end(v, h.ib, S, E);
        h.B = make_float3(fmaf(t, E.x - S.x, S.x), fmaf(t, E.y - S.y, S.y), fmaf(t, E.z - S.z, S.z));
        vertex_start_end(v, h.ic, S, E);
        h.C = make_float3(fmaf(t, E.x - S.x, S.x), fmaf(t, E.y - S.y, S.y), fmaf(t, E.z - S.z, S.z));
    }
    // barycentrics from the sheared edge functions of the watertight test
    const float ax = fmaf(-dx, h.A.z, h.A.x), ay = fmaf(-dy, h.A.z, h.A.y);
    const float bx = fmaf(-dx, h.B.z, h.B.x), by = fmaf(-dy, h.B.z, h.B.y);
    const float cx = fmaf(-dx, h.C.z, h.C.x), cy = fmaf(-dy, h.C.z, h.C.y);
    const float U = __fsub_rn(__fmul_rn(cx, by), __fmul_rn(cy, bx));
    const float V = __fsub_rn(__fmul_rn(ax, cy), __fmul_rn(ay, cx));
    const float W = __fsub_rn(__fmul_rn(bx, ay), __fmul_rn(by, ax));
    h.det = U + V + W;
    const float inv = h.det != 0.f ? 1.f / h.det : 0.f;
    h.inv_det = inv;
    h.b0 = U * inv;
    h.b1 = V * inv;
    h.b2 = W * inv;
    float3 n = cross3_rn(sub3(h.B, h.A), sub3(h.C, h.A));
    const float flip = dot3(n, h.dir) > 0.f ? -1.f : 1.f;
    const float nn = dot3(n, n);
    const float rs = nn > 0.f ? rsqrtf(nn) : 0.f;
    h.inl = flip * rs;
    h.n = scale3(n, h.inl);
    if ((kFeat & kFeatF64) && v.fp64) {
        const float sm = fmaxf(fabsf(ax) + fabsf(ay), fmaxf(fabsf(bx) + fabsf(by), fabsf(cx) + fabsf(cy)));
        const float zm = fmaxf(fabsf(h.A.z), fmaxf(fabsf(h.B.z), fabsf(h.C.z)));
        const float mag = zm * (1.f + fabsf(dx) + fabsf(dy)) + sm;
        if (2.f * kRelCoordShade * mag * sm > kBaryRel * fabsf(h.det))
            pixel_hit64(v, i, j, h);
    }
    float3 l = make_float3(fmaf(t, v.l1[0] - v.l0[0], v.l0[0]), fmaf(t, v.l1[1] - v.l0[1], v.l0[1]),
                           fmaf(t, v.l1[2] - v.l0[2], v.l0[2]));
    h.l = scale3(l, rsqrtf(dot3(l, l)));
    h.ndl = dot3(h.n, h.l);
    h.sigma = fmaf(v.k_d, fmaxf(h.ndl, 0.f), v.k_a);
    h.spec = 0.f;
    h.ndh = 0.f;
    if ((kFeat & kFeatSpec) && v.k_s > 0.f) {
        // the eye at the pixel time is the camera origin: v = -dir / |dir|
        const float3 e = scale3(h.dir, -rsqrtf(dot3(h.dir, h.dir)));
        const float3 hh = add3(h.l, e);
        h.hv = scale3(hh, rsqrtf(fmaxf(dot3(hh, hh), 1e-30f)));
        h.ndh = dot3(h.n, h.hv);
        h.spec = h.ndh > 0.f ? v.k_s * powf(h.ndh, v.shininess) : 0.f;
    }
}

__device__ __noinline__ void pixel_hit64(const ViewDev &v, int i, int j, PixelHit &h)
{
    const Ray64 ry = pixel_ray64(v, i, j);
    const double d[3] = {ry.dx, ry.dy, 1.0};
    const int vid[3] = {h.ia, h.ib, h.ic};
    double P[3][3];
    for (int k = 0; k < 3; ++k) {
        const float4 va = v.vtx[2 * vid[k]], vb = v.vtx[2 * vid[k] + 1];
        const double p[3] = {va.x, va.y, va.z}, e[3] = {p[0] + (double)va.w, p[1] + (double)vb.x, p[2] + (double)vb.y};
        for (int r = 0; r < 3; ++r) {
            const double S = (double)v.R0[3 * r] * p[0] + (double)v.R0[3 * r + 1] * p[1] + (double)v.R0[3 * r + 2] * p[2] +
                             (double)v.T0[r];
            const double E = (double)v.R1[3 * r] * e[0] + (double)v.R1[3 * r + 1] * e[1] + (double)v.R1[3 * r + 2] * e[2] +
                             (double)v.T1[r];
            P[k][r] = (1.0 - ry.t) * S + ry.t * E;
        }
    }
    double w[3];
    for (int k = 0; k < 3; ++k) {
        const double *b = P[(k + 1) % 3], *c = P[(k + 2) % 3];
        w[k] = d[0] * (b[1] * c[2] - b[2] * c[1]) + d[1] * (b[2] * c[0] - b[0] * c[2]) + d[2] * (b[0] * c[1] - b[1] * c[0]);
    }
    const double sw = w[0] + w[1] + w[2];
    if (sw != 0.0) {
        const double isw = 1.0 / sw;
        h.b0 = (float)(w[0] * isw);
        h.b1 = (float)(w[1] * isw);
        h.b2 = (float)(w[2] * isw);
        h.det = (float)(-sw);  // the watertight edge functions are -w
        h.inv_det = h.det != 0.f ? 1.f / h.det : 0.f;
    }
    const double e1[3] = {P[1][0] - P[0][0], P[1][1] - P[0][1], P[1][2] - P[0][2]};
    const double e2[3] = {P[2][0] - P[0][0], P[2][1] - P[0][1], P[2][2] - P[0][2]};
    const double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    const double nn = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
    if (nn > 0.0) {
        const double il = rsqrt(nn);
        const double s = n[0] * d[0] + n[1] * d[1] + n[2] * d[2] > 0.0 ? -il : il;
        h.n = make_float3((float)(n[0] * s), (float)(n[1] * s), (float)(n[2] * s));
        h.inl = (float)s;
    }
    h.A = make_float3((float)P[0][0], (float)P[0][1], (float)P[0][2]);
    h.B = make_float3((float)P[1][0], (float)P[1][1], (float)P[1][2]);
    h.C = make_float3((float)P[2][0], (float)P[2][1], (float)P[2][2]);
}

// Stages (d) and (e) run each warp over kShadeBlocks consecutive pixel
// blocks of kBlkW x kBlkH (8 x 4; lane -> column lane % kBlkW, row
// lane / kBlkW of each), so the lanes of a
// warp mostly see the same triangles: gathers of vertex data coalesce, and
// the adjoint sums a triangle's contributions over a lane's pixels and then
// over the warp before touching memory.  blk_offs[q] = first pixel block of
// view q in the batch.  One block per warp measured fastest on the stereo
// HMD frame (0.170 ms against 0.229 ms for two and 0.242 ms for four): the
// running sums held across pixels push the kernel into register spills
// that cost more than the warp reductions they save.
constexpr int kShadeBlocks = 1;

// CTAs of the shading kernels: 64 threads (two warps), 18 resident per SM,
// which caps them at 56 registers (36 warps per SM).  A CTA's slot frees
// only when its slowest warp finishes, and the warps of a CTA see different
// pixel blocks (background, one triangle, several), so small CTAs keep the
// SM fuller: 64 x 18 measured fastest against 256 x 4, 128 x 8, 128 x 9,
// 128 x 10, 64 x 16 and 32 x 32.
constexpr int kShadeThreads = 64, kShadeCtasPerSm = 18;

__device__ __forceinline__ bool block_pixel(const ViewDev *views, int nviews, const long long *blk_offs, long long b,
                                            int lane, int &q, long long &lin, int &i, int &j)
{
    q = find_view_warp(blk_offs, nviews, b);  // b is the warp's
    const ViewDev &v = views[q];
    const int lb = (int)(b - v.blk_off);  // < 2^23 blocks per view
    const int bw = (v.W + kBlkW - 1) / kBlkW;
    const int by = (int)(((unsigned long long)(unsigned)lb * v.bw_mul) >> 40);  // lb / bw
    i = (lb - by * bw) * kBlkW + lane % kBlkW;
    j = by * kBlkH + lane / kBlkW;
    lin = (long long)j * v.W + i;
    return i < v.W && j < v.H;
}

// Vertex colours of the visible triangle and the interpolated albedo
// a = sum_k b_k col_k of the pixel (shared by the shading and the adjoint).
struct PixelAlbedo {
    float col[3][3];  // [vertex][channel]
    float a[3];
};

__device__ __forceinline__ void pixel_albedo(const ViewDev &v, const PixelHit &h, PixelAlbedo &pa)
{
    const int vid[3] = {h.ia, h.ib, h.ic};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float4 c = v.col4[vid[k]];
        pa.col[k][0] = c.x;
        pa.col[k][1] = c.y;
        pa.col[k][2] = c.z;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
        pa.a[c] = fmaf(h.b0, pa.col[0][c], fmaf(h.b1, pa.col[1][c], h.b2 * pa.col[2][c]));
}

// Sums value l of every lane of `mask` over the warp and adds it to
// gradient l of the warp's triangle with vertices (v0, v1, v2): value 9k + c
// is d/dcol_k[c], 9k + 3 + c the sum of (1 - t) dL/dc_k[c] and 9k + 6 + c
// the sum of t dL/dc_k[c], with c_k the moved camera-space vertex k.  The
// position and velocity gradients follow once per triangle from the last
// two: dc/dp = (1-t) R0 + t R1 and dc/dv = t R1, so dL/dp = R0^T sum (1-t)
// dL/dc + R1^T sum t dL/dc and dL/dv = R1^T sum t dL/dc.  Lanes outside the
// group pass zeros.  Reduce-scatter: at each of five steps a lane keeps the
// half of its values selected by its lane bit and adds its partner's copy
// of that half, so lane l ends with the warp sum of value l (31 shuffles
// instead of 27 full butterflies).
__device__ __forceinline__ void reduce_add_triangle(const ViewDev &v, float (&s)[32], int v0, int v1, int v2)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int step = 0; step < 5; ++step) {
        const int half = 16 >> step;
        const bool upper = (lane & half) != 0;
#pragma unroll
        for (int k = 0; k < half; ++k) {
            const float send = upper ? s[k] : s[k + half];
            const float keep = upper ? s[k + half] : s[k];
            s[k] = keep + __shfl_xor_sync(0xffffffffu, send, half);
        }
    }
    const int k = min(lane / 9, 2), r = lane - 9 * k;
    const int base = 9 * k;
    const float o0 = __shfl_sync(0xffffffffu, s[0], base + 3), o1 = __shfl_sync(0xffffffffu, s[0], base + 4),
                o2 = __shfl_sync(0xffffffffu, s[0], base + 5);
    const float t0 = __shfl_sync(0xffffffffu, s[0], base + 6), t1 = __shfl_sync(0xffffffffu, s[0], base + 7),
                t2 = __shfl_sync(0xffffffffu, s[0], base + 8);
    if (lane < 27) {
        const int c = r < 3 ? r : (r < 6 ? r - 3 : r - 6);
        const int vk = k == 0 ? v0 : (k == 1 ? v1 : v2);
        float val = s[0];
        if (r >= 3) {
            val = fmaf(v.R1[c], t0, fmaf(v.R1[3 + c], t1, v.R1[6 + c] * t2));
            if (r < 6)
                val = fmaf(v.R0[c], o0, fmaf(v.R0[3 + c], o1, fmaf(v.R0[6 + c], o2, val)));
        }
        float *dst = r < 3 ? v.dcol : (r < 6 ? v.dpos : v.dvel);
        if (dst)
            atomicAdd(&dst[3 * vk + c], val);
    }
}

// Adjoint of rgb = a sigma + s, a = sum_k b_k col_k, sigma = k_a + k_d max(0, n.l),
// s = k_s max(0, n.h)^m (h depends only on the pixel's time and ray):
//  - d/dcol_k = g b_k sigma
//  - d/dn = (g . a) k_d l [n.l > 0] + (sum_c g_c) k_s m (n.h)^(m-1) h [n.h > 0]
//  - barycentrics b_k = w_k / sum w with w_0 = dir.(B x C), w_1 = dir.(C x A),
//    w_2 = dir.(A x B) (the watertight U, V, W are -w), so
//    d sum/dw_j = (gb_j - sum_k gb_k b_k) / sum w and dw_j/dA etc. are
//    cross products with dir;
//  - the unit normal n = flip (B-A)x(C-A) / |.|: dn gets (I - n n^T)/|.|;
//  - moved vertex c(t) = (1-t) S + t E with S = R0 p + T0, E = R1 (p + v) + T1
//    (applied per triangle after the warp sum, reduce_add_triangle).
// The pixel's 27 values (layout of reduce_add_triangle) are ADDED to acc.
template <int kFeat>
__device__ __forceinline__ void adjoint_add(const ViewDev &v, const PixelHit &h, const PixelAlbedo &pa, float g0,
                                            float g1, float g2, float (&acc)[27])
{
    {
        const float b[3] = {h.b0, h.b1, h.b2};
        const float gs[3] = {g0 * h.sigma, g1 * h.sigma, g2 * h.sigma};
        float gb[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
#pragma unroll
            for (int c = 0; c < 3; ++c)
                acc[9 * k + c] = fmaf(gs[c], b[k], acc[9 * k + c]);
            gb[k] = fmaf(gs[0], pa.col[k][0], fmaf(gs[1], pa.col[k][1], gs[2] * pa.col[k][2]));
        }
        const float gsig = fmaf(g0, pa.a[0], fmaf(g1, pa.a[1], g2 * pa.a[2]));
        // barycentrics -> moved vertices: with w_0 = D.(B x C) etc.,
        // dL/dA = gw1 (D x C) + gw2 (B x D) = D x (gw1 C - gw2 B), cyclically
        const float gdotb = fmaf(gb[0], b[0], fmaf(gb[1], b[1], gb[2] * b[2]));
        const float isw = -h.inv_det;  // 1 / sum w, sum w = -det (exactly the negated reciprocal)
        const float gw0 = (gb[0] - gdotb) * isw, gw1 = (gb[1] - gdotb) * isw, gw2 = (gb[2] - gdotb) * isw;
        const float3 D = h.dir;
        float3 gA = cross3(D, sub3(scale3(h.C, gw1), scale3(h.B, gw2)));
        float3 gB = cross3(D, sub3(scale3(h.A, gw2), scale3(h.C, gw0)));
        float3 gC = cross3(D, sub3(scale3(h.B, gw0), scale3(h.A, gw1)));
        // normal -> moved vertices: the diffuse term through n.l, the
        // specular term k_s (n.h)^m (white) through n.h; the three
        // contributions (B-C) x gn, (C-A) x gn, (A-B) x gn sum to zero
        const bool dif = h.ndl > 0.f, spc = (kFeat & kFeatSpec) && h.spec > 0.f;
        if ((dif || spc) && h.inl != 0.f) {
            float3 gnh = scale3(h.l, dif ? gsig * v.k_d : 0.f);
            if (spc)
                gnh = add3(gnh, scale3(h.hv, (g0 + g1 + g2) * v.shininess * h.spec / h.ndh));
            const float pr = dot3(h.n, gnh);
            const float3 gnn = scale3(sub3(gnh, scale3(h.n, pr)), h.inl);
            const float3 na = cross3(sub3(h.B, h.C), gnn), nb = cross3(sub3(h.C, h.A), gnn);
            gA = add3(gA, na);
            gB = add3(gB, nb);
            gC = sub3(gC, add3(na, nb));
        }
        // the moved vertices' gradients, split by the weights (1 - t) of S
        // and t of E
        const float3 gk[3] = {gA, gB, gC};
        const float t = h.t, omt = 1.f - t;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            acc[9 * k + 3] = fmaf(omt, gk[k].x, acc[9 * k + 3]);
            acc[9 * k + 4] = fmaf(omt, gk[k].y, acc[9 * k + 4]);
            acc[9 * k + 5] = fmaf(omt, gk[k].z, acc[9 * k + 5]);
            acc[9 * k + 6] = fmaf(t, gk[k].x, acc[9 * k + 6]);
            acc[9 * k + 7] = fmaf(t, gk[k].y, acc[9 * k + 7]);
            acc[9 * k + 8] = fmaf(t, gk[k].z, acc[9 * k + 8]);
        }
    }
}

// A lane's running sums of the adjoint values of the pixels it has seen
// since the last flush, all of one triangle of one view.
struct AdjointSum {
    float s[27];
    int q;  // view of the triangle (-1: nothing summed)
    unsigned id;
    int ia, ib, ic;
};

__device__ __forceinline__ void adjoint_reset(AdjointSum &a)
{
#pragma unroll
    for (int e = 0; e < 27; ++e)
        a.s[e] = 0.f;
    a.q = -1;
}

// Sums the lanes' running sums over the warp per distinct (view, triangle),
// adds them to the gradients and resets them.  Called by every lane.
__device__ __forceinline__ void adjoint_flush(const ViewDev *views, AdjointSum &a)
{
    unsigned rem = __ballot_sync(0xffffffffu, a.q >= 0);
    if (rem) {
        int leader = __ffs(rem) - 1;
        int tq = __shfl_sync(0xffffffffu, a.q, leader);
        unsigned tid = __shfl_sync(0xffffffffu, a.id, leader);
        float s[32];
        if (__all_sync(0xffffffffu, a.q < 0 || (a.q == tq && a.id == tid))) {
            // one triangle over the warp (the common case): lanes without
            // a sum hold zeros already
#pragma unroll
            for (int e = 0; e < 27; ++e)
                s[e] = a.s[e];
#pragma unroll
            for (int e = 27; e < 32; ++e)
                s[e] = 0.f;
            reduce_add_triangle(views[tq], s, __shfl_sync(0xffffffffu, a.ia, leader),
                                __shfl_sync(0xffffffffu, a.ib, leader), __shfl_sync(0xffffffffu, a.ic, leader));
        } else {
            while (true) {
                const bool mine = a.q == tq && a.id == tid;
                rem &= ~__ballot_sync(0xffffffffu, mine);
#pragma unroll
                for (int e = 0; e < 27; ++e)
                    s[e] = mine ? a.s[e] : 0.f;
#pragma unroll
                for (int e = 27; e < 32; ++e)
                    s[e] = 0.f;
                reduce_add_triangle(views[tq], s, __shfl_sync(0xffffffffu, a.ia, leader),
                                    __shfl_sync(0xffffffffu, a.ib, leader), __shfl_sync(0xffffffffu, a.ic, leader));
                if (!rem)
                    break;
                leader = __ffs(rem) - 1;
                tq = __shfl_sync(0xffffffffu, a.q, leader);
                tid = __shfl_sync(0xffffffffu, a.id, leader);
            }
        }
    }
    adjoint_reset(a);
}

// Adds a valid lane's pixel (triangle id of view q) to its running sum;
// first, if any lane's sum is of another triangle or view, the warp
// flushes.  Called by every lane.
template <int kFeat>
__device__ __forceinline__ void adjoint_step(const ViewDev *views, AdjointSum &a, bool valid, int q, unsigned id,
                                             const PixelHit &h, const PixelAlbedo &pa, float g0, float g1, float g2)
{
    if (__any_sync(0xffffffffu, valid && a.q >= 0 && (a.q != q || a.id != id)))
        adjoint_flush(views, a);
    if (valid) {
        adjoint_add<kFeat>(views[q], h, pa, g0, g1, g2, a.s);
        a.q = q;
        a.id = id;
        a.ia = h.ia;
        a.ib = h.ib;
        a.ic = h.ic;
    }
}

__device__ __forceinline__ bool frame_overflowed(const Counters *frame_cnt)
{
    return frame_cnt && (frame_cnt->status & (ST_OVERFLOW_PAIRS | ST_OVERFLOW_ITEMS | ST_OVERFLOW_FLAGS | ST_TIMEOUT));
}

// Stage (d).  keys != null: the frame's packed depth|id keys are resolved
// here too (id and depth written, then shaded), saving a separate resolve
// pass.  kAdjoint (a training frame): for views with a gradient input, the
// stage (e) adjoint of the pixel follows from the same PixelHit -- with an
// L2 target, from the colour just computed -- so the frame needs no
// separate adjoint pass.  Whole warps run (the adjoint's reductions).
// views: the device table, or the kernel's parameter table (k_shade_pv).
template <bool kAdjoint, int kFeat>
__device__ __forceinline__ void shade_body(const ViewDev *__restrict__ views, int nviews,
                                           const long long *__restrict__ blk_offs, long long nblocks,
                                           unsigned long long *__restrict__ keys, int reset_keys,
                                           const Counters *__restrict__ frame_cnt)
{
    const long long b0 = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * kShadeBlocks;
    if (b0 >= nblocks)
        return;  // whole warps
    const int lane = threadIdx.x & 31;
    // a training frame whose forward overflowed is rerun by the host: its
    // adjoint must not accumulate
    const bool adjoint = kAdjoint && !frame_overflowed(frame_cnt);
    AdjointSum acc;
    adjoint_reset(acc);
    for (int p = 0; p < kShadeBlocks && b0 + p < nblocks; ++p) {
        int q, pi, pj;
        long long lin;
        const bool inside = block_pixel(views, nviews, blk_offs, b0 + p, lane, q, lin, pi, pj);
        const ViewDev &v = views[q];
        const long long plane = (long long)v.W * v.H;
        const bool grad = adjoint && (v.grad_in || v.target || v.target_u8);
        // the upstream gradient (or L2 target) does not depend on the hit:
        // its loads go out first, before the key and the stores below
        float gin[3] = {0.f, 0.f, 0.f};
        if (grad && inside) {
            if (v.target_u8) {
                gin[0] = u8_unit(v.target_u8[lin]);
                gin[1] = u8_unit(v.target_u8[plane + lin]);
                gin[2] = u8_unit(v.target_u8[2 * plane + lin]);
            } else {
                const float *gsrc = v.grad_in ? v.grad_in : v.target;
                gin[0] = gsrc[lin];
                gin[1] = gsrc[plane + lin];
                gin[2] = gsrc[2 * plane + lin];
            }
        }
        unsigned id = 0xFFFFFFFFu;
        if (inside) {
            if (keys) {
                const unsigned long long key = keys[v.pix_off + lin];
                const bool bg = key == ~0ull;
                if (!bg && reset_keys)
                    keys[v.pix_off + lin] = ~0ull;  // left as the next frame wants it
                id = bg ? 0xFFFFFFFFu : (unsigned)(key & 0xFFFFFFFFull);
                if (v.id_out)
                    v.id_out[lin] = id;
                if (v.depth_out)
                    v.depth_out[lin] = bg ? INFINITY : __uint_as_float((unsigned)(key >> 32));
            } else {
                id = v.id_in[lin];
            }
        }
        // a view with neither an image nor a gradient only needs the resolve
        const bool hit = inside && id < (unsigned)v.T && (v.rgb_out || grad);
        PixelHit h;
        PixelAlbedo pa;
        float rgb[3] = {0.f, 0.f, 0.f};
        if (hit) {
            pixel_hit<kFeat>(v, pi, pj, id, h);
            pixel_albedo(v, h, pa);
            rgb[0] = fmaf(pa.a[0], h.sigma, h.spec);
            rgb[1] = fmaf(pa.a[1], h.sigma, h.spec);
            rgb[2] = fmaf(pa.a[2], h.sigma, h.spec);
        }
        if (inside && v.rgb_out) {
            v.rgb_out[lin] = rgb[0];
            v.rgb_out[plane + lin] = rgb[1];
            v.rgb_out[2 * plane + lin] = rgb[2];
        }
        if (kAdjoint) {
            const bool valid = hit && grad;
            float g0 = gin[0], g1 = gin[1], g2 = gin[2];
            float lsum = 0.f;  // this pixel's share of the L2 loss (background: rgb = 0)
            if (grad && inside && !v.grad_in) {
                // L2 loss sum (rgb - target)^2: its gradient from this frame's image
                const float e0 = rgb[0] - gin[0], e1 = rgb[1] - gin[1], e2 = rgb[2] - gin[2];
                lsum = fmaf(e0, e0, fmaf(e1, e1, e2 * e2));
                g0 = 2.f * e0;
                g1 = 2.f * e1;
                g2 = 2.f * e2;
            }
            adjoint_step<kFeat>(views, acc, valid, q, id, h, pa, g0, g1, g2);
            if (adjoint && v.loss) {
                // one view per warp: a warp sum, then one atomic into one of
                // the view's partial sums (one address for every warp of a
                // view would serialise them)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
                    lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
                if (lane == 0)
                    atomicAdd(&v.loss_part[(unsigned)b0 & (kLossSlots - 1)], lsum);
            }
        }
    }
    if (kAdjoint)
        adjoint_flush(views, acc);
}

template <bool kAdjoint, int kFeat>
__global__ void __launch_bounds__(kShadeThreads, kShadeCtasPerSm)
    k_shade(const ViewDev *__restrict__ views, int nviews, const long long *__restrict__ blk_offs, long long nblocks,
            unsigned long long *__restrict__ keys, int reset_keys, const Counters *__restrict__ frame_cnt)
{
    shade_body<kAdjoint, kFeat>(views, nviews, blk_offs, nblocks, keys, reset_keys, frame_cnt);
}

template <bool kAdjoint, int kFeat>
__global__ void __launch_bounds__(kShadeThreads, kShadeCtasPerSm)
    k_shade_pv(const __grid_constant__ ParamViews pv, int nviews, const long long *__restrict__ blk_offs,
               long long nblocks, unsigned long long *__restrict__ keys, int reset_keys,
               const Counters *__restrict__ frame_cnt)
{
    shade_body<kAdjoint, kFeat>(pv.v, nviews, blk_offs, nblocks, keys, reset_keys, frame_cnt);
}

// A training frame's losses: one block per view sums the view's partial
// sums and adds them to the caller's loss (views without a loss: nothing).
__global__ void __launch_bounds__(kLossSlots) k_loss_finalize(const ViewDev *__restrict__ views,
                                                              const Counters *__restrict__ frame_cnt)
{
    const ViewDev &v = views[blockIdx.x];
    if (!v.loss || frame_overflowed(frame_cnt))
        return;  // an overflowed forward is rerun by the host: its loss must not count
    float s = v.loss_part[threadIdx.x];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ float ws[kLossSlots / 32];
    if ((threadIdx.x & 31) == 0)
        ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < kLossSlots / 32; ++w)
            t += ws[w];
        atomicAdd(v.loss, t);  // several views may share one loss
    }
}

cudaError_t launch_loss_finalize(const ViewDev *views, int nviews, const Counters *frame_cnt, cudaStream_t st)
{
    if (nviews > 0)
        k_loss_finalize<<<nviews, kLossSlots, 0, st>>>(views, frame_cnt);
    return cudaGetLastError();
}

// Warps of kShadeBlocks blocks, kShadeThreads threads per CTA.
static unsigned shade_grid(long long nblocks)
{
    const long long warps = (nblocks + kShadeBlocks - 1) / kShadeBlocks;
    return (unsigned)((warps * 32 + kShadeThreads - 1) / kShadeThreads);
}

// The parameter table of a launch's views (null: the batch is too large, or
// the caller has no host copy; the kernels then read the device table).
static const ParamViews *param_views(const ViewDev *host_views, int nviews)
{
    static thread_local ParamViews pv;
    if (!host_views || nviews < 1 || nviews > kParamViews)
        return nullptr;
    std::memcpy(pv.v, host_views, sizeof(ViewDev) * (size_t)nviews);
    return &pv;
}

template <bool kAdjoint, int kFeat>
static void launch_shade_one(unsigned g, const ViewDev *views, const ParamViews *pv, int nviews,
                             const long long *blk_offs, long long nblocks, unsigned long long *keys, int reset_keys,
                             const Counters *frame_cnt, cudaStream_t st)
{
    if (pv)
        k_shade_pv<kAdjoint, kFeat><<<g, kShadeThreads, 0, st>>>(*pv, nviews, blk_offs, nblocks, keys, reset_keys,
                                                                 frame_cnt);
    else
        k_shade<kAdjoint, kFeat><<<g, kShadeThreads, 0, st>>>(views, nviews, blk_offs, nblocks, keys, reset_keys,
                                                              frame_cnt);
}

template <bool kAdjoint>
static void launch_shade_t(int feat, unsigned g, const ViewDev *views, const ParamViews *pv, int nviews,
                           const long long *blk_offs, long long nblocks, unsigned long long *keys, int reset_keys,
                           const Counters *frame_cnt, cudaStream_t st)
{
    if (feat == kFeatF64) {  // the precision form without the specular and sampled-foveation paths
        launch_shade_one<kAdjoint, kFeatF64>(g, views, pv, nviews, blk_offs, nblocks, keys, reset_keys, frame_cnt, st);
        return;
    }
    if (feat & kFeatF64) {  // the precision form with either: one variant with every path (same bits)
        launch_shade_one<kAdjoint, kFeatSpec | kFeatLut | kFeatF64>(g, views, pv, nviews, blk_offs, nblocks, keys,
                                                                    reset_keys, frame_cnt, st);
        return;
    }
    switch (feat) {
    case 0:
        launch_shade_one<kAdjoint, 0>(g, views, pv, nviews, blk_offs, nblocks, keys, reset_keys, frame_cnt, st);
        break;
    case kFeatSpec:
        launch_shade_one<kAdjoint, kFeatSpec>(g, views, pv, nviews, blk_offs, nblocks, keys, reset_keys, frame_cnt, st);
        break;
    case kFeatLut:
        launch_shade_one<kAdjoint, kFeatLut>(g, views, pv, nviews, blk_offs, nblocks, keys, reset_keys, frame_cnt, st);
        break;
    default:
        launch_shade_one<kAdjoint, kFeatSpec | kFeatLut>(g, views, pv, nviews, blk_offs, nblocks, keys, reset_keys,
                                                         frame_cnt, st);
    }
}

int shade_features(const ViewDev *vd, int n)
{
    int f = 0;
    for (int k = 0; k < n; ++k) {
        if (vd[k].k_s > 0.f)
            f |= kFeatSpec;
        if (vd[k].p_lut && (vd[k].mode == PR_FOVEATED || vd[k].mode == PR_BOTH))
            f |= kFeatLut;
        if (vd[k].fp64)
            f |= kFeatF64;
    }
    return f;
}

cudaError_t launch_shade(const ViewDev *views, int nviews, const long long *blk_offs, long long nblocks,
                         unsigned long long *keys, bool reset_keys, bool adjoint, const Counters *frame_cnt, int feat,
                         cudaStream_t st, const ViewDev *host_views)
{
    if (nblocks > 0) {
        const unsigned g = shade_grid(nblocks);
        const ParamViews *pv = param_views(host_views, nviews);
        if (adjoint)
            launch_shade_t<true>(feat, g, views, pv, nviews, blk_offs, nblocks, keys, reset_keys, frame_cnt, st);
        else
            launch_shade_t<false>(feat, g, views, pv, nviews, blk_offs, nblocks, keys, reset_keys, frame_cnt, st);
    }
    return cudaGetLastError();
}

// Stage (e) on its own: the adjoint of a shaded frame from its id buffer
// and an upstream gradient.
template <int kFeat>
__device__ __forceinline__ void backward_body(const ViewDev *__restrict__ views, int nviews,
                                              const long long *__restrict__ blk_offs, long long nblocks,
                                              const Counters *__restrict__ frame_cnt)
{
    const long long b0 = (((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * kShadeBlocks;
    if (b0 >= nblocks)
        return;  // whole warps
    // in a training frame: a forward that overflowed is rerun by the host,
    // so its adjoint must not accumulate
    if (frame_overflowed(frame_cnt))
        return;
    const int lane = threadIdx.x & 31;
    AdjointSum acc;
    adjoint_reset(acc);
    for (int p = 0; p < kShadeBlocks && b0 + p < nblocks; ++p) {
        int q, pi, pj;
        long long lin;
        const bool inside = block_pixel(views, nviews, blk_offs, b0 + p, lane, q, lin, pi, pj);
        const ViewDev &v = views[q];
        unsigned id = 0xFFFFFFFFu;
        if (inside && (v.grad_in || v.target))  // views of a batch without a gradient are skipped
            id = v.id_in[lin];
        const bool valid = id < (unsigned)v.T;
        PixelHit h;
        PixelAlbedo pa;
        float g0 = 0.f, g1 = 0.f, g2 = 0.f;
        if (valid) {
            const long long plane = (long long)v.W * v.H;
            pixel_hit<kFeat>(v, pi, pj, id, h);
            pixel_albedo(v, h, pa);
            if (v.target) {
                // L2 loss sum (rgb - target)^2: its gradient from this frame's image
                g0 = 2.f * (v.rgb_out[lin] - v.target[lin]);
                g1 = 2.f * (v.rgb_out[plane + lin] - v.target[plane + lin]);
                g2 = 2.f * (v.rgb_out[2 * plane + lin] - v.target[2 * plane + lin]);
            } else {
                g0 = v.grad_in[lin];
                g1 = v.grad_in[plane + lin];
                g2 = v.grad_in[2 * plane + lin];
            }
        }
        adjoint_step<kFeat>(views, acc, valid, q, id, h, pa, g0, g1, g2);
    }
    adjoint_flush(views, acc);
}

template <int kFeat>
__global__ void __launch_bounds__(kShadeThreads, kShadeCtasPerSm)
    k_backward(const ViewDev *__restrict__ views, int nviews, const long long *__restrict__ blk_offs, long long nblocks,
               const Counters *__restrict__ frame_cnt)
{
    backward_body<kFeat>(views, nviews, blk_offs, nblocks, frame_cnt);
}

template <int kFeat>
__global__ void __launch_bounds__(kShadeThreads, kShadeCtasPerSm)
    k_backward_pv(const __grid_constant__ ParamViews pv, int nviews, const long long *__restrict__ blk_offs,
                  long long nblocks, const Counters *__restrict__ frame_cnt)
{
    backward_body<kFeat>(pv.v, nviews, blk_offs, nblocks, frame_cnt);
}

template <int kFeat>
static void launch_backward_one(unsigned g, const ViewDev *views, const ParamViews *pv, int nviews,
                                const long long *blk_offs, long long nblocks, const Counters *frame_cnt,
                                cudaStream_t st)
{
    if (pv)
        k_backward_pv<kFeat><<<g, kShadeThreads, 0, st>>>(*pv, nviews, blk_offs, nblocks, frame_cnt);
    else
        k_backward<kFeat><<<g, kShadeThreads, 0, st>>>(views, nviews, blk_offs, nblocks, frame_cnt);
}

cudaError_t launch_backward(const ViewDev *views, int nviews, const long long *blk_offs, long long nblocks,
                            const Counters *frame_cnt, int feat, cudaStream_t st, const ViewDev *host_views)
{
    if (nblocks > 0) {
        const unsigned g = shade_grid(nblocks);
        const ParamViews *pv = param_views(host_views, nviews);
        if (feat & kFeatF64) {
            launch_backward_one<kFeatSpec | kFeatLut | kFeatF64>(g, views, pv, nviews, blk_offs, nblocks, frame_cnt, st);
            return cudaGetLastError();
        }
        switch (feat) {
        case 0:
            launch_backward_one<0>(g, views, pv, nviews, blk_offs, nblocks, frame_cnt, st);
            break;
        case kFeatSpec:
            launch_backward_one<kFeatSpec>(g, views, pv, nviews, blk_offs, nblocks, frame_cnt, st);
            break;
        case kFeatLut:
            launch_backward_one<kFeatLut>(g, views, pv, nviews, blk_offs, nblocks, frame_cnt, st);
            break;
        default:
            launch_backward_one<kFeatSpec | kFeatLut>(g, views, pv, nviews, blk_offs, nblocks, frame_cnt, st);
        }
    }
    return cudaGetLastError();
}

}  // namespace pr
