// pr_bound.cuh -- math of stage (a), the per-triangle space-time-fovea bound
// (Sec. 4).  Host+device so that the catch-up interval can be unit-tested
// on the CPU through pr_debug_catch_interval.
#pragma once

#include <math.h>

#include "pr_internal.cuh"

namespace pr {

__host__ __device__ inline float2 f2sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ inline float cross2(float2 a, float2 b) { return a.x * b.y - a.y * b.x; }

// ---------------------------------------------------------------------------
// Zenon's catch-up interval (Sec. 4.2.4), exact form.
//
// The rolling scan shows display location x at time r(x) = d . x.  A point
// c(t) of the moving triangle is met by the scan when t = r(proj(c(t))).
// Multiplying by 2 z(t) > 0 turns this into h(t) = 2 t z - kx X - ky Y - ks z
// = 0 with kx = d0/tanX, ky = d1/tanY, ks = d0 + d1, which is linear in the
// camera-space point and therefore, for fixed t, linear in the barycentrics:
// h(t, b) = sum_k b_k h_k(t), where h_k(t) = a t^2 + b t + c is the quadratic
// of vertex k (the paper's rational catch-up equation of Sec. 4.2.4 with the
// scan speed and the perspective divide written out).  Some point of the
// triangle is met at time t exactly when min_k h_k(t) <= 0 <= max_k h_k(t);
// that set only changes at roots of the h_k, so it is bounded by
// [t_min, t_max] = hull of {roots in [t_lo, t_hi]} plus the domain ends where
// the condition already holds.  Unlike the paper's closed form, this needs
// neither one catch per vertex nor a fixed root branch.
//
// S: camera-space vertices at t = 0, D: their motion over the frame (all
// points must have z > 0 over [t_lo, t_hi]).  Returns false when no point of
// the triangle is ever met by the scan.  FP32 with explicit tolerances: every
// root gets a margin of kEpsT, near-double roots contribute their vertex,
// and the end conditions are tested with an evaluation-error allowance.
// ---------------------------------------------------------------------------
__host__ __device__ inline bool catch_interval(const float3 S[3], const float3 D[3], float tan_x, float tan_y,
                                               float d0, float d1, float t_lo, float t_hi, float &tmin, float &tmax)
{
    const float kx = d0 / tan_x, ky = d1 / tan_y, ks = d0 + d1;
    float lo = INFINITY, hi = -INFINITY;
    bool lo_le = false, lo_ge = false, hi_le = false, hi_ge = false;
    bool finite = true;
    for (int k = 0; k < 3; ++k) {
        const float a = 2.f * D[k].z;
        const float b = 2.f * S[k].z - kx * D[k].x - ky * D[k].y - ks * D[k].z;
        const float c = -(kx * S[k].x + ky * S[k].y + ks * S[k].z);
        if (!(isfinite(a) && isfinite(b) && isfinite(c)))
            finite = false;
        // evaluation-error allowance of h at the domain ends
        const float m1 = 2.f * fabsf(S[k].z) + kx * fabsf(D[k].x) + ky * fabsf(D[k].y) + ks * fabsf(D[k].z);
        const float m0 = kx * fabsf(S[k].x) + ky * fabsf(S[k].y) + ks * fabsf(S[k].z);
        const float ends[2] = {t_lo, t_hi};
        for (int e = 0; e < 2; ++e) {
            const float t = ends[e];
            const float h = fmaf(fmaf(a, t, b), t, c);
            const float tol = 1e-5f * (fabsf(a) * t * t + m1 * fabsf(t) + m0) + 1e-30f;
            const bool le = h <= tol, ge = h >= -tol;
            if (e == 0) {
                lo_le |= le;
                lo_ge |= ge;
            } else {
                hi_le |= le;
                hi_ge |= ge;
            }
        }
        // roots
        float r[2];
        int nr = 0;
        const float scale = fabsf(b) + fabsf(c);
        if (fabsf(a) <= 1e-7f * scale) {
            if (b != 0.f)
                r[nr++] = -c / b;
        } else {
            const float disc = b * b - 4.f * a * c;
            const float dtol = 1e-5f * (b * b + 4.f * fabsf(a * c));
            if (disc < -dtol) {
            } else if (disc <= dtol) {
                r[nr++] = -b / (2.f * a);
            } else {
                const float q = -0.5f * (b + copysignf(sqrtf(disc), b));
                r[nr++] = q / a;
                if (q != 0.f)
                    r[nr++] = c / q;
            }
        }
        for (int e = 0; e < nr; ++e) {
            if (r[e] >= t_lo - kEpsT && r[e] <= t_hi + kEpsT) {
                lo = fminf(lo, r[e] - kEpsT);
                hi = fmaxf(hi, r[e] + kEpsT);
            }
        }
    }
    if (!finite) {
        tmin = t_lo;
        tmax = t_hi;
        return true;
    }
    if (lo_le && lo_ge)
        lo = t_lo;
    if (hi_le && hi_ge)
        hi = t_hi;
    lo = fmaxf(lo, t_lo);
    hi = fminf(hi, t_hi);
    if (!(lo <= hi))
        return false;
    tmin = lo;
    tmax = hi;
    return true;
}

// Bounding box (x0, x1, y0, y1) of the annular sector around f between the
// unit directions a (clockwise end) and b (counter-clockwise end, less than
// half a turn from a) and the radii [rho0, rho1]; full = the whole disc.
__host__ __device__ inline float4 sector_box(float2 f, float2 a, float2 b, float rho0, float rho1, bool full)
{
    if (full)
        return make_float4(f.x - rho1, f.x + rho1, f.y - rho1, f.y + rho1);
    float x0 = INFINITY, x1 = -INFINITY, y0 = INFINITY, y1 = -INFINITY;
    const float2 c[4] = {make_float2(f.x + rho0 * a.x, f.y + rho0 * a.y), make_float2(f.x + rho0 * b.x, f.y + rho0 * b.y),
                         make_float2(f.x + rho1 * a.x, f.y + rho1 * a.y), make_float2(f.x + rho1 * b.x, f.y + rho1 * b.y)};
    for (int k = 0; k < 4; ++k) {
        x0 = fminf(x0, c[k].x);
        x1 = fmaxf(x1, c[k].x);
        y0 = fminf(y0, c[k].y);
        y1 = fmaxf(y1, c[k].y);
    }
    const float2 ax[4] = {make_float2(1.f, 0.f), make_float2(0.f, 1.f), make_float2(-1.f, 0.f), make_float2(0.f, -1.f)};
    for (int k = 0; k < 4; ++k) {
        if (cross2(a, ax[k]) >= 0.f && cross2(ax[k], b) >= 0.f) {
            x0 = fminf(x0, f.x + rho1 * ax[k].x);
            x1 = fmaxf(x1, f.x + rho1 * ax[k].x);
            y0 = fminf(y0, f.y + rho1 * ax[k].y);
            y1 = fmaxf(y1, f.y + rho1 * ax[k].y);
        }
    }
    return make_float4(x0, x1, y0, y1);
}

// Rotate the unit vector a by the small angle whose sine is sn (positive =
// counter-clockwise).
__host__ __device__ inline float2 rot_small(float2 a, float sn)
{
    sn = fminf(fmaxf(sn, -1.f), 1.f);
    const float cs = sqrtf(fmaxf(0.f, 1.f - sn * sn));
    return make_float2(a.x * cs - a.y * sn, a.x * sn + a.y * cs);
}

// Display box (x0, x1, y0, y1) that contains q of the framebuffer box
// [u0,u1] x [v0,v1]: the same sector argument with the radius map p (the
// power map of alpha, or the sampled p when lut is set).
__host__ __device__ inline float4 fov_image_box(float u0, float u1, float v0, float v1, float2 f, float alpha,
                                                const float *lut = nullptr, int n = 0)
{
    const float2 c[4] = {make_float2(u0, v0), make_float2(u1, v0), make_float2(u1, v1), make_float2(u0, v1)};
    float rmax = 0.f;
    for (int k = 0; k < 4; ++k) {
        const float2 w = f2sub(c[k], f);
        rmax = fmaxf(rmax, sqrtf(w.x * w.x + w.y * w.y));
    }
    const SampledP sp{lut, n};
    const float kD1 = powf(kSqrt2, 1.f - alpha);
    const float rho1 = (lut ? sp.p(rmax) : kD1 * powf(rmax, alpha)) * (1.f + 1e-5f) + 1e-7f;
    const bool inside = f.x >= u0 && f.x <= u1 && f.y >= v0 && f.y <= v1;
    if (inside)
        return sector_box(f, make_float2(1.f, 0.f), make_float2(1.f, 0.f), 0.f, rho1, true);
    const float cx = fminf(fmaxf(f.x, u0), u1), cy = fminf(fmaxf(f.y, v0), v1);
    const float rmin = sqrtf((cx - f.x) * (cx - f.x) + (cy - f.y) * (cy - f.y));
    const float rho0 = (lut ? sp.p(rmin) : kD1 * powf(rmin, alpha)) * (1.f - 1e-5f);
    float2 a = f2sub(c[0], f), b = a;
    for (int k = 1; k < 4; ++k) {
        const float2 w = f2sub(c[k], f);
        if (cross2(a, w) < 0.f)
            a = w;
        if (cross2(b, w) > 0.f)
            b = w;
    }
    const float la = sqrtf(a.x * a.x + a.y * a.y), lb = sqrtf(b.x * b.x + b.y * b.y);
    a = rot_small(make_float2(a.x / la, a.y / la), -1e-6f);
    b = rot_small(make_float2(b.x / lb, b.y / lb), 1e-6f);
    return sector_box(f, a, b, rho0, rho1, false);
}

}  // namespace pr
