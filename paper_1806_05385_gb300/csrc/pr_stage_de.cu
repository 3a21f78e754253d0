// pr_stage_de.cu -- stage (d): deferred shading at the pixel time (Sec. 3.2,
// "Shading"), and stage (e): its adjoint with respect to the vertex colours,
// positions and velocities, with the visible triangle of every pixel held
// fixed.  Both recompute the pixel's time, ray, moved triangle and
// barycentrics from the id buffer instead of storing them.
#include "pr_launch.h"

namespace pr {

__device__ __forceinline__ float3 sub3(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ float3 cross3(float3 a, float3 b)
{
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 scale3(float3 a, float s) { return make_float3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float3 add3(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }

// Everything shading needs about the visible triangle at one pixel.
struct PixelHit {
    int ia, ib, ic;     // vertex indices
    float t;            // pixel time
    float3 dir;         // ray direction
    float3 A, B, C;     // triangle moved to t (camera space)
    float b0, b1, b2;   // barycentrics of the ray point
    float det;          // U + V + W of the watertight test
    float3 n;           // unit normal facing the viewer
    float nlen, flip;   // |(B-A) x (C-A)| and the sign applied
    float3 l;           // unit light direction at t
    float ndl, sigma;   // n.l and k_a + k_d max(0, n.l)
    float3 hv;          // Blinn-Phong half vector normalize(l + v), v = the reversed ray
    float ndh, spec;    // n.h and k_s max(0, n.h)^shininess (0 without specular)
};

__device__ __forceinline__ void pixel_hit(const ViewDev &v, int i, int j, unsigned id, PixelHit &h)
{
    float x0, x1, dx, dy;
    pixel_ray(v, i, j, x0, x1, h.t, dx, dy);
    h.dir = make_float3(dx, dy, 1.f);
    h.ia = v.i0[id];
    h.ib = v.i1[id];
    h.ic = v.i2[id];
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
    h.b0 = U * inv;
    h.b1 = V * inv;
    h.b2 = W * inv;
    float3 n = cross3(sub3(h.B, h.A), sub3(h.C, h.A));
    h.flip = dot3(n, h.dir) > 0.f ? -1.f : 1.f;
    const float nn = dot3(n, n);
    const float rs = nn > 0.f ? rsqrtf(nn) : 0.f;
    h.nlen = nn * rs;
    const float in = h.flip * rs;
    h.n = scale3(n, in);
    float3 l = make_float3(fmaf(t, v.l1[0] - v.l0[0], v.l0[0]), fmaf(t, v.l1[1] - v.l0[1], v.l0[1]),
                           fmaf(t, v.l1[2] - v.l0[2], v.l0[2]));
    h.l = scale3(l, rsqrtf(dot3(l, l)));
    h.ndl = dot3(h.n, h.l);
    h.sigma = v.k_a + v.k_d * fmaxf(h.ndl, 0.f);
    h.spec = 0.f;
    h.ndh = 0.f;
    if (v.k_s > 0.f) {
        // the eye at the pixel time is the camera origin: v = -dir / |dir|
        const float3 e = scale3(h.dir, -rsqrtf(dot3(h.dir, h.dir)));
        const float3 hh = add3(h.l, e);
        h.hv = scale3(hh, rsqrtf(fmaxf(dot3(hh, hh), 1e-30f)));
        h.ndh = dot3(h.n, h.hv);
        h.spec = h.ndh > 0.f ? v.k_s * powf(h.ndh, v.shininess) : 0.f;
    }
}

// Stages (d) and (e) run one warp per 8x4 pixel block (lane -> column
// lane % 8, row lane / 8), so the lanes of a warp mostly see the same
// triangles: gathers of vertex data coalesce and the adjoint can sum a
// triangle's contributions over the warp before touching memory.
// blk_offs[q] = first 8x4 block of view q in the batch.
__device__ __forceinline__ bool block_pixel(const ViewDev *views, int nviews, const long long *blk_offs, long long g,
                                            const ViewDev *&vp, long long &lin, int &i, int &j)
{
    const long long b = g >> 5;
    const int lane = (int)(g & 31);
    const ViewDev &v = views[find_view(blk_offs, nviews, b)];
    vp = &v;
    const int lb = (int)(b - v.blk_off);  // < 2^23 blocks per view: 32-bit division
    const int bw = (v.W + 7) >> 3;
    const int by = lb / bw;
    i = (lb - by * bw) * 8 + (lane & 7);
    j = by * 4 + (lane >> 3);
    lin = (long long)j * v.W + i;
    return i < v.W && j < v.H;
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
//  - moved vertex c(t) = (1-t) S + t E with S = R0 p + T0, E = R1 (p + v) + T1:
//    dc/dp = (1-t) R0 + t R1, dc/dv = t R1.
// Per warp, the 27 contributions of each distinct triangle are summed over
// the lanes that see it with a reduce-scatter (lane l ends with the sum of
// value l) and added with one 27-lane atomic instruction.  Called by every
// lane of a warp; valid = this lane has a pixel with a visible triangle.
__device__ __forceinline__ void adjoint_pixel(const ViewDev &v, const PixelHit &h, bool valid, unsigned id, float g0,
                                              float g1, float g2)
{
    float gc[3][3], gp[3][3], gvel[3][3];
    int vid[3] = {0, 0, 0};
    for (int k = 0; k < 3; ++k)
        for (int c = 0; c < 3; ++c)
            gc[k][c] = gp[k][c] = gvel[k][c] = 0.f;
    if (valid) {
        vid[0] = h.ia;
        vid[1] = h.ib;
        vid[2] = h.ic;
        const float b[3] = {h.b0, h.b1, h.b2};
        float col[3][3];
        for (int k = 0; k < 3; ++k) {
            col[k][0] = v.cr[vid[k]];
            col[k][1] = v.cg[vid[k]];
            col[k][2] = v.cb[vid[k]];
        }
        float a[3];
        for (int c = 0; c < 3; ++c)
            a[c] = b[0] * col[0][c] + b[1] * col[1][c] + b[2] * col[2][c];
        float gb[3];
        const float gv[3] = {g0, g1, g2};
        for (int k = 0; k < 3; ++k) {
            gb[k] = 0.f;
            for (int c = 0; c < 3; ++c) {
                gc[k][c] = gv[c] * b[k] * h.sigma;
                gb[k] += gv[c] * col[k][c];
            }
            gb[k] *= h.sigma;
        }
        const float gsig = g0 * a[0] + g1 * a[1] + g2 * a[2];
        // barycentrics -> moved vertices
        const float sw = -h.det;
        const float gdotb = gb[0] * b[0] + gb[1] * b[1] + gb[2] * b[2];
        const float isw = sw != 0.f ? 1.f / sw : 0.f;
        const float gw0 = (gb[0] - gdotb) * isw, gw1 = (gb[1] - gdotb) * isw, gw2 = (gb[2] - gdotb) * isw;
        const float3 D = h.dir;
        float3 gA = add3(scale3(cross3(D, h.C), gw1), scale3(cross3(h.B, D), gw2));
        float3 gB = add3(scale3(cross3(h.C, D), gw0), scale3(cross3(D, h.A), gw2));
        float3 gC = add3(scale3(cross3(D, h.B), gw0), scale3(cross3(h.A, D), gw1));
        // normal -> moved vertices: the diffuse term through n.l, the
        // specular term k_s (n.h)^m (white) through n.h
        const bool dif = h.ndl > 0.f, spc = h.spec > 0.f;
        if ((dif || spc) && h.nlen > 0.f) {
            float3 gnh = scale3(h.l, dif ? gsig * v.k_d : 0.f);
            if (spc)
                gnh = add3(gnh, scale3(h.hv, (g0 + g1 + g2) * v.shininess * h.spec / h.ndh));
            const float pr = dot3(h.n, gnh);
            const float3 gnn = scale3(sub3(gnh, scale3(h.n, pr)), h.flip / h.nlen);
            gA = add3(gA, cross3(sub3(h.B, h.C), gnn));
            gB = add3(gB, cross3(sub3(h.C, h.A), gnn));
            gC = add3(gC, cross3(sub3(h.A, h.B), gnn));
        }
        // moved vertices -> positions and velocities
        const float3 gk[3] = {gA, gB, gC};
        const float t = h.t, omt = 1.f - t;
        for (int k = 0; k < 3; ++k) {
            for (int c = 0; c < 3; ++c) {
                const float e1 = v.R1[c] * gk[k].x + v.R1[3 + c] * gk[k].y + v.R1[6 + c] * gk[k].z;
                gp[k][c] = omt * (v.R0[c] * gk[k].x + v.R0[3 + c] * gk[k].y + v.R0[6 + c] * gk[k].z) + t * e1;
                gvel[k][c] = t * e1;
            }
        }
    }
    const int lane = threadIdx.x & 31;
    unsigned rem = __ballot_sync(0xffffffffu, valid);
    while (rem) {
        const int leader = __ffs(rem) - 1;
        const unsigned tid = __shfl_sync(0xffffffffu, id, leader);
        const bool mine = valid && id == tid;
        rem &= ~__ballot_sync(0xffffffffu, mine);
        // the 27 contributions of this triangle (value 9k + c: colour,
        // 9k + 3 + c: position, 9k + 6 + c: velocity of vertex k), zero for
        // lanes that see another triangle, padded to 32
        float s[32];
#pragma unroll
        for (int k = 0; k < 3; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                s[9 * k + c] = mine ? gc[k][c] : 0.f;
                s[9 * k + 3 + c] = mine ? gp[k][c] : 0.f;
                s[9 * k + 6 + c] = mine ? gvel[k][c] : 0.f;
            }
#pragma unroll
        for (int e = 27; e < 32; ++e)
            s[e] = 0.f;
        // reduce-scatter over the warp: at each step a lane keeps the half
        // of its values selected by its lane bit and adds its partner's
        // copy of that half; after five steps lane l holds the warp sum of
        // value l (31 shuffles instead of 27 full butterflies)
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
        const int k = lane / 9, r = lane - 9 * (lane / 9);
        const int v0 = __shfl_sync(0xffffffffu, vid[0], leader), v1 = __shfl_sync(0xffffffffu, vid[1], leader),
                  v2 = __shfl_sync(0xffffffffu, vid[2], leader);
        if (lane < 27) {
            const int vk = k == 0 ? v0 : (k == 1 ? v1 : v2);
            float *dst = r < 3 ? v.dcol : (r < 6 ? v.dpos : v.dvel);
            if (dst)
                atomicAdd(&dst[3 * vk + (r % 3)], s[0]);
        }
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
template <bool kAdjoint>
__global__ void __launch_bounds__(256, 4) k_shade(const ViewDev *__restrict__ views, int nviews,
                                              const long long *__restrict__ blk_offs, long long nthreads,
                                              const unsigned long long *__restrict__ keys,
                                              const Counters *__restrict__ frame_cnt)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if ((g & ~31ll) >= nthreads)
        return;
    const ViewDev *vp = views;
    long long lin = 0;
    int pi = 0, pj = 0;
    const bool inside = g < nthreads && block_pixel(views, nviews, blk_offs, g, vp, lin, pi, pj);
    const ViewDev &v = *vp;
    unsigned id = 0xFFFFFFFFu;
    if (inside) {
        if (keys) {
            const unsigned long long key = keys[v.pix_off + lin];
            const bool bg = key == ~0ull;
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
    const bool hit = inside && id < (unsigned)v.T && (v.rgb_out || (kAdjoint && (v.grad_in || v.target)));
    const long long plane = (long long)v.W * v.H;
    PixelHit h;
    float rgb[3] = {0.f, 0.f, 0.f};
    if (hit) {
        pixel_hit(v, pi, pj, id, h);
        const float r = fmaf(h.b0, v.cr[h.ia], fmaf(h.b1, v.cr[h.ib], h.b2 * v.cr[h.ic]));
        const float gg = fmaf(h.b0, v.cg[h.ia], fmaf(h.b1, v.cg[h.ib], h.b2 * v.cg[h.ic]));
        const float b = fmaf(h.b0, v.cb[h.ia], fmaf(h.b1, v.cb[h.ib], h.b2 * v.cb[h.ic]));
        rgb[0] = fmaf(r, h.sigma, h.spec);
        rgb[1] = fmaf(gg, h.sigma, h.spec);
        rgb[2] = fmaf(b, h.sigma, h.spec);
    }
    if (inside && v.rgb_out) {
        v.rgb_out[lin] = rgb[0];
        v.rgb_out[plane + lin] = rgb[1];
        v.rgb_out[2 * plane + lin] = rgb[2];
    }
    if (kAdjoint) {
        // views of a batch without a gradient skip it (a warp covers one view)
        if (!(v.grad_in || v.target) || frame_overflowed(frame_cnt))
            return;
        float g0 = 0.f, g1 = 0.f, g2 = 0.f;
        if (hit) {
            if (v.target) {
                // L2 loss sum (rgb - target)^2: its gradient from this frame's image
                g0 = 2.f * (rgb[0] - v.target[lin]);
                g1 = 2.f * (rgb[1] - v.target[plane + lin]);
                g2 = 2.f * (rgb[2] - v.target[2 * plane + lin]);
            } else {
                g0 = v.grad_in[lin];
                g1 = v.grad_in[plane + lin];
                g2 = v.grad_in[2 * plane + lin];
            }
        }
        adjoint_pixel(v, h, hit, id, g0, g1, g2);
    }
}

cudaError_t launch_shade(const ViewDev *views, int nviews, const long long *blk_offs, long long nblocks,
                         const unsigned long long *keys, bool adjoint, const Counters *frame_cnt, cudaStream_t st)
{
    const long long n = nblocks * 32;
    if (n > 0) {
        if (adjoint)
            k_shade<true><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(views, nviews, blk_offs, n, keys, frame_cnt);
        else
            k_shade<false><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(views, nviews, blk_offs, n, keys, frame_cnt);
    }
    return cudaGetLastError();
}

// Stage (e) on its own: the adjoint of a shaded frame from its id buffer
// and an upstream gradient.
__global__ void __launch_bounds__(256, 4) k_backward(const ViewDev *__restrict__ views, int nviews,
                                                 const long long *__restrict__ blk_offs, long long nthreads,
                                                 const Counters *__restrict__ frame_cnt)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if ((g & ~31ll) >= nthreads)
        return;  // whole warps only
    // in a training frame: a forward that overflowed is rerun by the host,
    // so its adjoint must not accumulate
    if (frame_overflowed(frame_cnt))
        return;
    const ViewDev *vp = views;
    long long lin = 0;
    int pi = 0, pj = 0;
    const bool inside = g < nthreads && block_pixel(views, nviews, blk_offs, g, vp, lin, pi, pj);
    const ViewDev &v = *vp;
    if (!(v.grad_in || v.target))
        return;  // views of a batch without a gradient (a warp covers one view)
    unsigned id = 0xFFFFFFFFu;
    if (inside)
        id = v.id_in[lin];
    const bool valid = inside && id < (unsigned)v.T;
    PixelHit h;
    float g0 = 0.f, g1 = 0.f, g2 = 0.f;
    if (valid) {
        const long long plane = (long long)v.W * v.H;
        pixel_hit(v, pi, pj, id, h);
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
    adjoint_pixel(v, h, valid, id, g0, g1, g2);
}

cudaError_t launch_backward(const ViewDev *views, int nviews, const long long *blk_offs, long long nblocks,
                            const Counters *frame_cnt, cudaStream_t st)
{
    const long long n = nblocks * 32;
    if (n > 0)
        k_backward<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(views, nviews, blk_offs, n, frame_cnt);
    return cudaGetLastError();
}

}  // namespace pr
