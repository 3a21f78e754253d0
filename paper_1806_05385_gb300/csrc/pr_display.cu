// pr_display.cu -- the display step after shading (Sec. 3.1.1, "Display"):
// the foveated framebuffer image I_f becomes the display image
// I_u(x) = I_f(q^-1(x)).  Two methods, as in the paper:
//
//  - MIP + cubic: a MIP pyramid of I_f (2x2 box averages, sizes halved
//    with ceil, blocks cut by the border averaged over their texels) is
//    sampled tri-linearly at the level of detail of the largest stretch of
//    q^-1 at x times the size ratio, each level with a 3-tap cubic filter
//    (the nearest texel and its two neighbours per axis, cubic B-spline
//    weights normalised by their sum, clamped to the edge);
//  - projected 5x5: the framebuffer pixel that holds q^-1(x) and its 5x5
//    neighbourhood, weighted by a Gaussian reconstruction filter of the
//    display-space distance between x and q of each pixel centre,
//    normalised (the paper's projection of the display's reconstruction
//    filter into the foveated domain); weights are taken relative to the
//    nearest sample, whose factor cancels, so they cannot all underflow.
//
// One thread per display pixel; planar rgb in and out, coalesced along x.
#include <algorithm>
#include <cstring>

#include "pr_launch.h"

namespace pr {

constexpr int kMaxMipLevels = 16;  // 16384 x 16384 needs 15

struct MipPyramid {
    const float *lev[kMaxMipLevels];
    int w[kMaxMipLevels], h[kMaxMipLevels];
    int L;
};

// Display-step constants of a view (by value into the kernel).
struct DisplayView {
    int W, H, Wd, Hd;
    int fov;             // foveated or joint mode: q is the power map, else the identity
    float fx, fy;        // fovea
    float alpha, inv_alpha;
    const float *p_lut;  // or: the sampled p (then alpha is unused)
    int p_n;
    float scale;         // max(W / Wd, H / Hd)
    float sigma;         // projected filter width, display pixels
};

// Texel (x, y) of a level from the level below (w0 x h0): the 2x2 block's
// mean, over the texels of the block that exist.
__device__ __forceinline__ void mip_texel(const float *__restrict__ src, int w0, int h0, float *__restrict__ dst,
                                          int w1, int h1, int x, int y)
{
    const int x0 = 2 * x, y0 = 2 * y;
    const bool xr = x0 + 1 < w0, yr = y0 + 1 < h0;
    const float n = (float)((1 + xr) * (1 + yr));
    for (int c = 0; c < 3; ++c) {
        const float *s = src + (size_t)c * w0 * h0;
        float a = s[(size_t)y0 * w0 + x0];
        if (xr)
            a += s[(size_t)y0 * w0 + x0 + 1];
        if (yr) {
            a += s[(size_t)(y0 + 1) * w0 + x0];
            if (xr)
                a += s[(size_t)(y0 + 1) * w0 + x0 + 1];
        }
        dst[(size_t)c * w1 * h1 + (size_t)y * w1 + x] = a / n;
    }
}

__global__ void k_mip_down(const float *__restrict__ src, int w0, int h0, float *__restrict__ dst, int w1, int h1)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= w1 || y >= h1)
        return;
    mip_texel(src, w0, h0, dst, w1, h1, x, y);
}

// Display location q(c) of every framebuffer pixel centre c (the offset from
// the fovea scaled by (|e|/D)^(alpha - 1)), for the projected filter.
__device__ __forceinline__ float2 q_of(int W, int H, int fov, float fx, float fy, float alpha,
                                       const float *__restrict__ p_lut, int p_n, int i, int j)
{
    float q0 = __fdiv_rn((float)i + 0.5f, (float)W), q1 = __fdiv_rn((float)j + 0.5f, (float)H);
    if (fov) {
        const float e0 = q0 - fx, e1 = q1 - fy, r = sqrtf(fmaf(e0, e0, e1 * e1));
        const SampledP sp{p_lut, p_n};
        const float s = r > 0.f ? (p_lut ? sp.p(r) / r : powf(r * (1.f / kSqrt2), alpha - 1.f)) : 0.f;
        q0 = fmaf(e0, s, fx);
        q1 = fmaf(e1, s, fy);
    }
    return make_float2(q0, q1);
}

__device__ __forceinline__ void q_entry(int W, int H, int fov, float fx, float fy, float alpha,
                                        const float *__restrict__ p_lut, int p_n, float2 *__restrict__ table, int i,
                                        int j)
{
    table[(size_t)j * W + i] = q_of(W, H, fov, fx, fy, alpha, p_lut, p_n, i, j);
}

__global__ void k_q_table(int W, int H, int fov, float fx, float fy, float alpha, const float *__restrict__ p_lut,
                          int p_n, float2 *__restrict__ table)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
    if (i >= W)
        return;
    q_entry(W, H, fov, fx, fy, alpha, p_lut, p_n, table, i, j);
}

__device__ __forceinline__ float bspline3(float x)
{
    x = fabsf(x);
    if (x < 1.f)
        return fmaf(0.5f * x, x * x, 2.f / 3.f - x * x);
    if (x < 2.f) {
        const float y = 2.f - x;
        return y * y * y * (1.f / 6.f);
    }
    return 0.f;
}

// 3-tap cubic sample of one level at texel coordinates (s, t).
__device__ __forceinline__ void sample3(const float *__restrict__ lev, int w, int h, float s, float t, float out[3])
{
    const float fs = floorf(s + 0.5f), ft = floorf(t + 0.5f);
    float wx[3], wy[3], sx = 0.f, sy = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        wx[k] = bspline3(s - (fs + (float)(k - 1)));
        wy[k] = bspline3(t - (ft + (float)(k - 1)));
        sx += wx[k];
        sy += wy[k];
    }
    const float inv = 1.f / (sx * sy);
    out[0] = out[1] = out[2] = 0.f;
    const int is = (int)fs, it = (int)ft;
    const size_t plane = (size_t)w * h;
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
        const int y = min(max(it + ky - 1, 0), h - 1);
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
            const int x = min(max(is + kx - 1, 0), w - 1);
            const float wgt = wx[kx] * wy[ky] * inv;
            const size_t o = (size_t)y * w + x;
            out[0] = fmaf(wgt, __ldg(lev + o), out[0]);
            out[1] = fmaf(wgt, __ldg(lev + plane + o), out[1]);
            out[2] = fmaf(wgt, __ldg(lev + 2 * plane + o), out[2]);
        }
    }
}

// Display pixel (a, b) of a view.
template <int kMethod>
__device__ __forceinline__ void unfoveate_pixel(const DisplayView &dv, const MipPyramid &pyr,
                                                const float *__restrict__ rgb, const float2 *__restrict__ qtab,
                                                float *__restrict__ out, int a, int b)
{
    const float x0 = __fdiv_rn((float)a + 0.5f, (float)dv.Wd), x1 = __fdiv_rn((float)b + 0.5f, (float)dv.Hd);
    // u = q^-1(x): the offset from the fovea scaled by (|e|/D)^(1/alpha - 1)
    float u0 = x0, u1 = x1, tang = 1.f, stretch = 1.f;
    if (dv.fov) {
        const float e0 = x0 - dv.fx, e1 = x1 - dv.fy, r = sqrtf(fmaf(e0, e0, e1 * e1));
        if (dv.p_lut) {  // the sampled p: tangential stretch p^-1(r)/r, radial the slope of p^-1
            const SampledP sp{dv.p_lut, dv.p_n};
            const float radial = sp.dpinv(r);
            tang = r > 0.f ? sp.pinv(r) / r : radial;
            stretch = fmaxf(tang, radial);
        } else {
            tang = r > 0.f ? powf(r * (1.f / kSqrt2), dv.inv_alpha - 1.f) : INFINITY;
            stretch = fmaxf(tang, tang * dv.inv_alpha);
        }
        const float s = r > 0.f ? tang : 0.f;
        u0 = fmaf(e0, s, dv.fx);
        u1 = fmaf(e1, s, dv.fy);
    }
    float res[3];
    if (kMethod == PR_UNFOVEATE_MIP_CUBIC) {
        // level of detail: the largest stretch of q^-1 (tangential for alpha >= 1)
        float lambda = log2f(stretch * dv.scale);
        lambda = fminf(fmaxf(lambda, 0.f), (float)(pyr.L - 1));  // NaN-free: tang >= 0
        const int k0 = (int)floorf(lambda), k1 = min(k0 + 1, pyr.L - 1);
        const float f = lambda - (float)k0;
        float s0[3], s1[3];
        sample3(pyr.lev[k0], pyr.w[k0], pyr.h[k0], fmaf(u0, (float)pyr.w[k0], -0.5f),
                fmaf(u1, (float)pyr.h[k0], -0.5f), s0);
        if (f > 0.f) {
            sample3(pyr.lev[k1], pyr.w[k1], pyr.h[k1], fmaf(u0, (float)pyr.w[k1], -0.5f),
                    fmaf(u1, (float)pyr.h[k1], -0.5f), s1);
            for (int c = 0; c < 3; ++c)
                res[c] = fmaf(f, s1[c] - s0[c], s0[c]);
        } else {
            for (int c = 0; c < 3; ++c)
                res[c] = s0[c];
        }
    } else {
        const int i = min(max((int)floorf(u0 * (float)dv.W), 0), dv.W - 1);
        const int j = min(max((int)floorf(u1 * (float)dv.H), 0), dv.H - 1);
        const float k2 = -0.5f / (dv.sigma * dv.sigma);
        const size_t plane = (size_t)dv.W * dv.H;
        // display location q(c) of a window pixel's centre, from the table
        auto qc = [&](int pi, int pj, float &q0, float &q1) {
            const float2 q = __ldg(qtab + (size_t)pj * dv.W + pi);
            q0 = q.x;
            q1 = q.y;
        };
        // pass 1: the nearest sample in display space
        float d2min = INFINITY, qm0 = 0.f, qm1 = 0.f;
        for (int dy = -2; dy <= 2; ++dy)
            for (int dx = -2; dx <= 2; ++dx) {
                const int pi = i + dx, pj = j + dy;
                if (pj < 0 || pj >= dv.H || pi < 0 || pi >= dv.W)
                    continue;
                float q0, q1;
                qc(pi, pj, q0, q1);
                const float d0 = (x0 - q0) * (float)dv.Wd, d1 = (x1 - q1) * (float)dv.Hd;
                const float q2 = fmaf(d0, d0, d1 * d1);
                if (q2 < d2min) {
                    d2min = q2;
                    qm0 = q0;
                    qm1 = q1;
                }
            }
        // pass 2: weights relative to the nearest sample (its factor cancels
        // in the normalisation, so they never all underflow), with
        // d^2 - d_min^2 = (d - d_min)(d + d_min) per axis, where d - d_min
        // comes from the difference of the two samples' display locations
        float acc[3] = {0.f, 0.f, 0.f}, wsum = 0.f;
        for (int dy = -2; dy <= 2; ++dy)
            for (int dx = -2; dx <= 2; ++dx) {
                const int pi = i + dx, pj = j + dy;
                if (pj < 0 || pj >= dv.H || pi < 0 || pi >= dv.W)
                    continue;
                float q0, q1;
                qc(pi, pj, q0, q1);
                const float a0 = (qm0 - q0) * (float)dv.Wd, a1 = (qm1 - q1) * (float)dv.Hd;  // d - d_min
                const float b0 = (2.f * x0 - q0 - qm0) * (float)dv.Wd, b1 = (2.f * x1 - q1 - qm1) * (float)dv.Hd;
                const float w = expf(k2 * fmaf(a0, b0, a1 * b1));
                const size_t o = (size_t)pj * dv.W + pi;
                wsum += w;
                acc[0] = fmaf(w, __ldg(rgb + o), acc[0]);
                acc[1] = fmaf(w, __ldg(rgb + plane + o), acc[1]);
                acc[2] = fmaf(w, __ldg(rgb + 2 * plane + o), acc[2]);
            }
        const float inv = 1.f / wsum;
        for (int c = 0; c < 3; ++c)
            res[c] = acc[c] * inv;
    }
    const size_t dplane = (size_t)dv.Wd * dv.Hd, o = (size_t)b * dv.Wd + a;
    out[o] = res[0];
    out[dplane + o] = res[1];
    out[2 * dplane + o] = res[2];
}

template <int kMethod>
__global__ void __launch_bounds__(256) k_unfoveate(DisplayView dv, MipPyramid pyr, const float *__restrict__ rgb,
                                                  const float2 *__restrict__ qtab, float *__restrict__ out)
{
    const int a = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (a >= dv.Wd)
        return;
    unfoveate_pixel<kMethod>(dv, pyr, rgb, qtab, out, a, b);
}

// ---- the batched display step (MIP): many views, one launch per pyramid
// level and one for the display pixels of all views.  A launch's blocks are
// numbered view after view (blk[q] = first block of view q, blk[n] = all);
// a block finds its view by a binary search and runs the same per-texel and
// per-pixel code as the single-view kernels, so the results are the same.
struct DisplayBatchView {
    DisplayView dv;
    MipPyramid pyr;  // level 0 = rgb
    const float *rgb;
    float *out;
};

// The view of block b (the same for every lane): the warp compares 32
// offsets at a time (find_view_warp).  Called by whole warps.
__device__ __forceinline__ int block_view(const long long *__restrict__ blk, int n, long long b)
{
    return find_view_warp(blk, n, b);
}

// Level k of every view that has one (blocks of 256 texels, row-major).
__global__ void __launch_bounds__(256) k_mip_down_batch(const DisplayBatchView *__restrict__ tab,
                                                       const long long *__restrict__ blk, int n, int k)
{
    const int q = block_view(blk, n, blockIdx.x);
    const MipPyramid &pyr = tab[q].pyr;
    const int t = (int)(blockIdx.x - blk[q]) * (int)blockDim.x + (int)threadIdx.x;
    const int w1 = pyr.w[k], h1 = pyr.h[k];
    if (t >= w1 * h1)
        return;
    const int y = t / w1, x = t - y * w1;
    // levels k >= 1 live in the call's scratch (only level 0, the caller's
    // image, is read-only)
    mip_texel(pyr.lev[k - 1], pyr.w[k - 1], pyr.h[k - 1], const_cast<float *>(pyr.lev[k]), w1, h1, x, y);
}

// The display pixels of every view (blocks of 256, row-major; a view has
// fewer than 2^28 pixels, so its pixel index is 32-bit).  The register cap
// keeps the single-view kernel's occupancy (5 CTAs per SM): the view's
// constants, parameters there, are registers here.
__global__ void __launch_bounds__(256, 5) k_unfoveate_mip_batch(const DisplayBatchView *__restrict__ tab,
                                                               const long long *__restrict__ blk, int n)
{
    const int q = block_view(blk, n, blockIdx.x);
    const DisplayBatchView &e = tab[q];
    const DisplayView dv = e.dv;
    const int t = (int)(blockIdx.x - blk[q]) * (int)blockDim.x + (int)threadIdx.x;
    if (t >= dv.Wd * dv.Hd)
        return;
    const int b = t / dv.Wd, a = t - b * dv.Wd;
    unfoveate_pixel<PR_UNFOVEATE_MIP_CUBIC>(dv, e.pyr, e.rgb, nullptr, e.out, a, b);
}

int mip_level_count(int W, int H)
{
    int L = 1;
    while (W > 1 || H > 1) {
        W = (W + 1) / 2;
        H = (H + 1) / 2;
        ++L;
    }
    return L;
}

// Scratch floats of the display step: the MIP pyramid, or the q table of
// the projected filter (2 per framebuffer pixel).
size_t mip_pyramid_floats(int W, int H)
{
    size_t n = 0;
    for (;;) {
        n += (size_t)3 * W * H;
        if (W == 1 && H == 1)
            return n;
        W = (W + 1) / 2;
        H = (H + 1) / 2;
    }
}

cudaError_t launch_unfoveate(int method, int W, int H, int mode, float fx, float fy, float alpha, const float *p_lut,
                             int p_n, int Wd, int Hd, float sigma, const float *rgb, float *pyramid, float *out,
                             cudaStream_t st)
{
    DisplayView dv;
    dv.W = W;
    dv.H = H;
    dv.Wd = Wd;
    dv.Hd = Hd;
    dv.fov = mode == PR_FOVEATED || mode == PR_BOTH;
    dv.fx = fx;
    dv.fy = fy;
    dv.alpha = alpha;
    dv.inv_alpha = 1.f / alpha;
    dv.p_lut = p_lut;
    dv.p_n = p_n;
    dv.scale = fmaxf((float)W / (float)Wd, (float)H / (float)Hd);
    dv.sigma = sigma;
    MipPyramid pyr;
    std::memset(&pyr, 0, sizeof pyr);
    const dim3 blk(256), grd((unsigned)((Wd + 255) / 256), (unsigned)Hd);
    if (method == PR_UNFOVEATE_MIP_CUBIC) {
        const int L = mip_level_count(W, H);
        if (L > kMaxMipLevels)
            return cudaErrorInvalidValue;
        pyr.L = L;
        pyr.lev[0] = rgb;
        pyr.w[0] = W;
        pyr.h[0] = H;
        float *p = pyramid;
        for (int k = 1; k < L; ++k) {
            const int w1 = (pyr.w[k - 1] + 1) / 2, h1 = (pyr.h[k - 1] + 1) / 2;
            const dim3 b2(32, 8), g2((unsigned)((w1 + 31) / 32), (unsigned)((h1 + 7) / 8));
            k_mip_down<<<g2, b2, 0, st>>>(pyr.lev[k - 1], pyr.w[k - 1], pyr.h[k - 1], p, w1, h1);
            pyr.lev[k] = p;
            pyr.w[k] = w1;
            pyr.h[k] = h1;
            p += (size_t)3 * w1 * h1;
        }
        k_unfoveate<PR_UNFOVEATE_MIP_CUBIC><<<grd, blk, 0, st>>>(dv, pyr, rgb, nullptr, out);
    } else {
        float2 *qtab = reinterpret_cast<float2 *>(pyramid);
        const dim3 gq((unsigned)((W + 255) / 256), (unsigned)H);
        k_q_table<<<gq, 256, 0, st>>>(W, H, dv.fov, fx, fy, alpha, p_lut, p_n, qtab);
        k_unfoveate<PR_UNFOVEATE_PROJECTED><<<grd, blk, 0, st>>>(dv, pyr, rgb, qtab, out);
    }
    return cudaGetLastError();
}

static size_t view_scratch_floats(int W, int H)
{
    return (mip_pyramid_floats(W, H) + 3) & ~(size_t)3;  // 16-byte aligned carve
}

static size_t qtab_floats(int W, int H)
{
    return ((size_t)2 * W * H + 3) & ~(size_t)3;
}

size_t display_batch_scratch_floats(int method, const DisplayEntry *e, int n)
{
    size_t f = 0;
    for (int q = 0; q < n; ++q) {
        if (method == PR_UNFOVEATE_MIP_CUBIC)
            f += view_scratch_floats(e[q].W, e[q].H);  // every view's pyramid, side by side
        else
            f = std::max(f, qtab_floats(e[q].W, e[q].H));  // one view's q table at a time
    }
    return f;
}

// Table layout (MIP): n DisplayBatchView, then kMaxMipLevels arrays of n + 1
// block offsets: the display pixels' at index 0, pyramid level k's at k.
size_t display_batch_table_bytes(int n)
{
    const size_t views = ((sizeof(DisplayBatchView) * (size_t)n) + 15) & ~(size_t)15;
    return views + sizeof(long long) * (size_t)kMaxMipLevels * (size_t)(n + 1);
}

cudaError_t launch_unfoveate_batch(int method, float sigma, const DisplayEntry *e, int n, float *scratch,
                                   void *h_table, void *d_table, cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    if (method == PR_UNFOVEATE_PROJECTED) {
        // view after view with the single-view kernels (q table, then the
        // filter), each view's q table in the same scratch: the table of all
        // views at once, or of L2-sized groups, was measured slower
        for (int q = 0; q < n; ++q) {
            const cudaError_t err = launch_unfoveate(method, e[q].W, e[q].H, e[q].mode, e[q].fx, e[q].fy, e[q].alpha,
                                                     e[q].p_lut, e[q].p_n, e[q].Wd, e[q].Hd, sigma, e[q].rgb, scratch,
                                                     e[q].out, st);
            if (err != cudaSuccess)
                return err;
        }
        return cudaSuccess;
    }
    const size_t views_bytes = ((sizeof(DisplayBatchView) * (size_t)n) + 15) & ~(size_t)15;
    DisplayBatchView *tab = static_cast<DisplayBatchView *>(h_table);
    long long *blk = reinterpret_cast<long long *>(static_cast<char *>(h_table) + views_bytes);
    int Lmax = 1;
    float *p = scratch;
    for (int q = 0; q < n; ++q) {
        DisplayBatchView &t = tab[q];
        std::memset(&t, 0, sizeof t);
        DisplayView &dv = t.dv;
        dv.W = e[q].W;
        dv.H = e[q].H;
        dv.Wd = e[q].Wd;
        dv.Hd = e[q].Hd;
        dv.fov = e[q].mode == PR_FOVEATED || e[q].mode == PR_BOTH;
        dv.fx = e[q].fx;
        dv.fy = e[q].fy;
        dv.alpha = e[q].alpha;
        dv.inv_alpha = 1.f / e[q].alpha;
        dv.p_lut = e[q].p_lut;
        dv.p_n = e[q].p_n;
        dv.scale = fmaxf((float)dv.W / (float)dv.Wd, (float)dv.H / (float)dv.Hd);
        dv.sigma = sigma;
        t.rgb = e[q].rgb;
        t.out = e[q].out;
        // the view's scratch: its pyramid levels 1..
        float *lp = p;
        p += view_scratch_floats(dv.W, dv.H);
        const int L = mip_level_count(dv.W, dv.H);
        if (L > kMaxMipLevels)
            return cudaErrorInvalidValue;
        t.pyr.L = L;
        t.pyr.lev[0] = e[q].rgb;
        t.pyr.w[0] = dv.W;
        t.pyr.h[0] = dv.H;
        for (int k = 1; k < L; ++k) {
            t.pyr.w[k] = (t.pyr.w[k - 1] + 1) / 2;
            t.pyr.h[k] = (t.pyr.h[k - 1] + 1) / 2;
            t.pyr.lev[k] = lp;
            lp += (size_t)3 * t.pyr.w[k] * t.pyr.h[k];
        }
        Lmax = std::max(Lmax, L);
    }
    for (int k = 0; k < kMaxMipLevels; ++k) {
        long long *o = blk + (size_t)k * (n + 1);
        o[0] = 0;
        for (int q = 0; q < n; ++q) {
            const long long items = k == 0 ? (long long)tab[q].dv.Wd * tab[q].dv.Hd
                                           : (k < tab[q].pyr.L ? (long long)tab[q].pyr.w[k] * tab[q].pyr.h[k] : 0ll);
            o[q + 1] = o[q] + (items + 255) / 256;
        }
    }
    cudaError_t err = cudaMemcpyAsync(d_table, h_table, display_batch_table_bytes(n), cudaMemcpyHostToDevice, st);
    if (err != cudaSuccess)
        return err;
    const DisplayBatchView *dtab = static_cast<const DisplayBatchView *>(d_table);
    const long long *dblk = reinterpret_cast<const long long *>(static_cast<const char *>(d_table) + views_bytes);
    for (int k = 1; k < Lmax; ++k) {
        const long long nb = blk[(size_t)k * (n + 1) + n];
        if (nb > 0)
            k_mip_down_batch<<<(unsigned)nb, 256, 0, st>>>(dtab, dblk + (size_t)k * (n + 1), n, k);
    }
    if (blk[n] > 0)
        k_unfoveate_mip_batch<<<(unsigned)blk[n], 256, 0, st>>>(dtab, dblk, n);
    return cudaGetLastError();
}

}  // namespace pr
