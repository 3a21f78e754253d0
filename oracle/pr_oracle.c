/*
 * pr_oracle.c -- FP64 CPU oracle for perceptual rasterization
 * (Ritschel, Friston, Steed: "Perceptual Rasterization for Head-mounted
 * Display Image Synthesis", 2018).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, obviously correct
 * definition that the CUDA path is checked against.  Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg may load it; the library
 * and its kernels never call it, and it shares no code with them.
 *
 * What it computes (Sec. 3, "a correct, but slow, solution would be to test
 * all primitives against all pixels"; Sec. 5.2: perceptual rasterization is
 * identical to ray tracing every pixel at its own time):
 *
 *   for every requested framebuffer pixel (i, j):
 *     u   = ((i + 1/2) / W, (j + 1/2) / H)            unit framebuffer location
 *     x   = q(u) when foveated, else u                 display location (Sec. 3.1.1)
 *     t   = r(x) = x . d when rolling, else 0          pixel time (Sec. 3.1.2)
 *     dir = ((2 x0 - 1) tanX, (2 x1 - 1) tanY, 1)      camera-space ray, origin 0
 *     for EVERY triangle (no bounds, no tiles):
 *       move its camera-space vertices to time t      (Sec. 3.2, "Intersection")
 *       solve ray/plane + barycentrics by Cramer's rule in FP64
 *       hit if all barycentrics >= 0 and ray parameter s > z_near
 *     winner = lexicographic minimum of (s, triangle id)  (z-buffering, Sec. 3.2)
 *
 * Readings of the paper taken here:
 *  - q maps a framebuffer (foveated-image) location to its display location:
 *    q(u) = x_f + (u - x_f)/|u - x_f| * p(|u - x_f|), p(d) = D (d/D)^alpha,
 *    D = sqrt(2) (the domain of p in Sec. 3.1.1), so p(D) = D and alpha = 1
 *    is the identity.  The display samples I_f(q^-1(x)) (Sec. 3.1.1,
 *    "Display"), which fixes this direction.
 *  - in the joint mode the time is taken at the display location q(u)
 *    (Sec. 3.1.3 and Sec. 4.3: r o q).
 *  - vertex at time t: c(t) = (1-t) (R0 p + T0) + t (R1 (p + v) + T1), the
 *    linear interpolation of the start and end camera-space vertices M_s v_s
 *    and M_e v_e (Sec. 3.2, "Bounding" and "Intersection").
 *  - depth = the ray parameter s = camera z of the hit ("actual z value",
 *    Sec. 3.2), edges inclusive, ties broken by the smaller triangle id,
 *    no back-face culling.
 *  - shading (Sec. 3.2, "Shading": light is interpolated at the pixel time;
 *    not affected by foveation): Lambert with albedo a = sum_k b_k col_k,
 *    face normal of the moved triangle turned to face the viewer, light
 *    l(t) = normalize((1-t) R0 l_w + t R1 l_w), rgb = a (k_a + k_d max(0, n.l))
 *    + k_s max(0, n.h)^shininess with the rolling specular half vector
 *    h = normalize(l(t) + v), v = the reversed ray (the eye at the pixel
 *    time is the camera origin; "Rolling Shading", Sec. 6).
 *
 * Build: plain C99 + OpenMP, -ffp-contract=off so that x86 and Arm give the
 * same bits.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    double tan_x, tan_y, z_near;
    double pose0[16], pose1[16]; /* row-major world->camera, at t = 0 and t = 1 */
    double fovea[2];             /* x_f in unit framebuffer coordinates */
    double alpha;                /* p(d) = D (d/D)^alpha */
    double d[2];                 /* rolling skew direction, r(x) = x . d */
    double light_w[3];           /* world-space unit direction towards the light */
    double k_a, k_d;             /* ambient and diffuse weights */
    double k_s, shininess;       /* rolling specular (Blinn-Phong): weight (0: none) and exponent */
    int32_t W, H;
    int32_t mode;                /* 0 classic, 1 rolling, 2 foveated, 3 both */
    int32_t p_n;                 /* > 0: p is given by p_lut[0..p_n] instead of the power map */
    const double *p_lut;         /* p at d_k = k D / p_n (increasing, p_lut[0] = 0) */
} or_view;

enum { OR_CLASSIC = 0, OR_ROLLING = 1, OR_FOVEATED = 2, OR_BOTH = 3 };

static const double OR_D = 1.4142135623730950488; /* sqrt(2) */

/* ---------------------------------------------------------------- foveation */

/* p(d) = D (d/D)^alpha: maps a framebuffer distance from the fovea to a
 * display distance (Sec. 3.1.1, power foveation of Sec. 5.1). */
double or_p(double dist, double alpha) { return OR_D * pow(dist / OR_D, alpha); }

/* p^-1(r) = D (r/D)^(1/alpha). */
double or_pinv(double r, double alpha) { return OR_D * pow(r / OR_D, 1.0 / alpha); }

/* An arbitrary monotone p (Sec. 3.1.1: "any monotonic p"), given by its
 * values at d_k = k D / n: linear between the samples (the last segment
 * continued beyond D), and p^-1 its exact inverse (the segment that holds r,
 * inverted; the paper's numerical inversion). */
static double lut_p(const or_view *v, double d)
{
    const int64_t n = v->p_n;
    const double x = d * (double)n / OR_D;
    int64_t k = (int64_t)floor(x);
    if (k < 0)
        k = 0;
    if (k > n - 1)
        k = n - 1;
    const double t = x - (double)k;
    return (1.0 - t) * v->p_lut[k] + t * v->p_lut[k + 1];
}

static int64_t lut_segment(const or_view *v, double r)
{
    int64_t lo = 0, hi = v->p_n - 1; /* last k with p_lut[k] <= r */
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) / 2;
        if (v->p_lut[mid] <= r)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

static double lut_pinv(const or_view *v, double r)
{
    const int64_t k = lut_segment(v, r);
    const double a = v->p_lut[k], b = v->p_lut[k + 1];
    return ((double)k + (r - a) / (b - a)) * OR_D / (double)v->p_n;
}

/* d p^-1 / dr at r (the slope of the segment that holds it). */
static double lut_dpinv(const or_view *v, double r)
{
    const int64_t k = lut_segment(v, r);
    return OR_D / (double)v->p_n / (v->p_lut[k + 1] - v->p_lut[k]);
}

static double view_p(const or_view *v, double d) { return v->p_n > 0 ? lut_p(v, d) : or_p(d, v->alpha); }
static double view_pinv(const or_view *v, double r) { return v->p_n > 0 ? lut_pinv(v, r) : or_pinv(r, v->alpha); }

/* q: framebuffer -> display, radial about the fovea (Sec. 3.1.1). */
void or_q(const or_view *v, const double u[2], double x[2])
{
    double e0 = u[0] - v->fovea[0], e1 = u[1] - v->fovea[1];
    double dist = sqrt(e0 * e0 + e1 * e1);
    if (dist == 0.0) {
        x[0] = v->fovea[0];
        x[1] = v->fovea[1];
        return;
    }
    double s = view_p(v, dist) / dist;
    x[0] = v->fovea[0] + e0 * s;
    x[1] = v->fovea[1] + e1 * s;
}

/* q^-1: display -> framebuffer, q with p^-1 in place of p (Sec. 3.1.1). */
void or_qinv(const or_view *v, const double x[2], double u[2])
{
    double e0 = x[0] - v->fovea[0], e1 = x[1] - v->fovea[1];
    double dist = sqrt(e0 * e0 + e1 * e1);
    if (dist == 0.0) {
        u[0] = v->fovea[0];
        u[1] = v->fovea[1];
        return;
    }
    double s = view_pinv(v, dist) / dist;
    u[0] = v->fovea[0] + e0 * s;
    u[1] = v->fovea[1] + e1 * s;
}

/* ---------------------------------------------------------------- pixel ray */

/* Time, display location and camera-space ray direction of pixel (i, j). */
void or_pixel(const or_view *v, int64_t i, int64_t j, double *t, double x[2], double dir[3])
{
    double u[2] = {(i + 0.5) / v->W, (j + 0.5) / v->H};
    int foveated = (v->mode == OR_FOVEATED || v->mode == OR_BOTH);
    int rolling = (v->mode == OR_ROLLING || v->mode == OR_BOTH);
    if (foveated)
        or_q(v, u, x);
    else {
        x[0] = u[0];
        x[1] = u[1];
    }
    *t = rolling ? (x[0] * v->d[0] + x[1] * v->d[1]) : 0.0;
    dir[0] = (2.0 * x[0] - 1.0) * v->tan_x;
    dir[1] = (2.0 * x[1] - 1.0) * v->tan_y;
    dir[2] = 1.0;
}

/* --------------------------------------------------------------- vertices */

static void xform(const double M[16], const double p[3], double out[3])
{
    for (int r = 0; r < 3; ++r)
        out[r] = M[4 * r + 0] * p[0] + M[4 * r + 1] * p[1] + M[4 * r + 2] * p[2] + M[4 * r + 3];
}

/* Camera-space start and end positions of one vertex: S = M_s v_s and
 * E = M_e v_e with v_s = p and v_e = p + v (Sec. 3.2, "Bounding"). */
static void vertex_start_end(const or_view *v, const double *pos, const double *vel, int64_t k,
                             double S[3], double E[3])
{
    double ps[3] = {pos[3 * k], pos[3 * k + 1], pos[3 * k + 2]};
    double pe[3] = {ps[0] + vel[3 * k], ps[1] + vel[3 * k + 1], ps[2] + vel[3 * k + 2]};
    xform(v->pose0, ps, S);
    xform(v->pose1, pe, E);
}

/* Vertex at time t: linear interpolation of its start and end positions. */
static void lerp3(const double S[3], const double E[3], double t, double out[3])
{
    for (int r = 0; r < 3; ++r)
        out[r] = (1.0 - t) * S[r] + t * E[r];
}

/* -------------------------------------------------------- ray / triangle */

static double det3(const double a[3], const double b[3], const double c[3])
{
    /* determinant of the 3x3 matrix with columns a, b, c */
    return a[0] * (b[1] * c[2] - b[2] * c[1]) - b[0] * (a[1] * c[2] - a[2] * c[1]) +
           c[0] * (a[1] * b[2] - a[2] * b[1]);
}

/* Ray from the origin along dir against triangle (A, B, C) by Cramer's rule
 * on  [B-A, C-A, -dir] (b1, b2, s)^T = -A.  Writes the barycentrics of A, B,
 * C and the ray parameter s (NaN-free only when the system is regular).
 * Returns 1 when the system is regular. */
static int cramer(const double A[3], const double B[3], const double C[3], const double dir[3],
                  double b[3], double *s)
{
    double e1[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
    double e2[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
    double nd[3] = {-dir[0], -dir[1], -dir[2]};
    double rhs[3] = {-A[0], -A[1], -A[2]};
    double det = det3(e1, e2, nd);
    if (det == 0.0) {
        b[0] = b[1] = b[2] = -1.0;
        *s = INFINITY;
        return 0;
    }
    b[1] = det3(rhs, e2, nd) / det;
    b[2] = det3(e1, rhs, nd) / det;
    *s = det3(e1, e2, rhs) / det;
    b[0] = 1.0 - b[1] - b[2];
    return 1;
}

static int is_hit(int regular, const double b[3], double s, double z_near)
{
    return regular && b[0] >= 0.0 && b[1] >= 0.0 && b[2] >= 0.0 && s > z_near;
}

static void tri_at(const or_view *v, const double *pos, const double *vel, const int32_t *tri,
                   int64_t id, double t, double P[3][3])
{
    for (int k = 0; k < 3; ++k) {
        double S[3], E[3];
        vertex_start_end(v, pos, vel, tri[3 * id + k], S, E);
        lerp3(S, E, t, P[k]);
    }
}

/* ---------------------------------------------------------------- shading */

static void cross(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Camera-space unit light direction at time t (rolling shading, Sec. 3.2). */
void or_light(const or_view *v, double t, double l[3])
{
    double l0[3], l1[3];
    for (int r = 0; r < 3; ++r) {
        l0[r] = v->pose0[4 * r] * v->light_w[0] + v->pose0[4 * r + 1] * v->light_w[1] + v->pose0[4 * r + 2] * v->light_w[2];
        l1[r] = v->pose1[4 * r] * v->light_w[0] + v->pose1[4 * r + 1] * v->light_w[1] + v->pose1[4 * r + 2] * v->light_w[2];
    }
    for (int r = 0; r < 3; ++r)
        l[r] = (1.0 - t) * l0[r] + t * l1[r];
    double n = sqrt(dot(l, l));
    for (int r = 0; r < 3; ++r)
        l[r] /= n;
}

/* Unit face normal of (A, B, C), turned to face the viewer (n . dir <= 0);
 * also returns the unnormalised normal length and the flip sign. */
static void face_normal(const double P[3][3], const double dir[3], double nh[3], double *len, double *flip)
{
    double e1[3] = {P[1][0] - P[0][0], P[1][1] - P[0][1], P[1][2] - P[0][2]};
    double e2[3] = {P[2][0] - P[0][0], P[2][1] - P[0][1], P[2][2] - P[0][2]};
    double n[3];
    cross(e1, e2, n);
    *flip = dot(n, dir) > 0.0 ? -1.0 : 1.0;
    *len = sqrt(dot(n, n));
    for (int r = 0; r < 3; ++r)
        nh[r] = *flip * n[r] / *len;
}

/* Rolling specular (Blinn-Phong, "Rolling Shading" of Sec. 6): the eye at
 * the pixel time is the camera origin, so the unit vector from the hit to
 * the eye is the reversed ray; h = normalize(l + v).  Returns n . h. */
static double half_vector(const double l[3], const double dir[3], const double nh[3], double hv[3])
{
    const double dn = sqrt(dot(dir, dir));
    for (int r = 0; r < 3; ++r)
        hv[r] = l[r] - dir[r] / dn;
    const double hn = sqrt(dot(hv, hv));
    for (int r = 0; r < 3; ++r)
        hv[r] /= hn;
    return dot(nh, hv);
}

static void shade(const or_view *v, const double P[3][3], const double b[3], const double *col,
                  const int32_t *vid, double t, const double dir[3], double rgb[3])
{
    double nh[3], len, flip, l[3], hv[3];
    face_normal(P, dir, nh, &len, &flip);
    or_light(v, t, l);
    double ndl = dot(nh, l);
    double sigma = v->k_a + v->k_d * (ndl > 0.0 ? ndl : 0.0);
    double spec = 0.0;
    if (v->k_s > 0.0) {
        const double ndh = half_vector(l, dir, nh, hv);
        spec = ndh > 0.0 ? v->k_s * pow(ndh, v->shininess) : 0.0;
    }
    for (int c = 0; c < 3; ++c) {
        double a = b[0] * col[3 * vid[0] + c] + b[1] * col[3 * vid[1] + c] + b[2] * col[3 * vid[2] + c];
        rgb[c] = a * sigma + spec;
    }
}

/* ----------------------------------------------------------------- render */

/*
 * Render the pixels listed in pix[0..npix) (linear index j*W + i), or every
 * pixel when pix == NULL (then npix must be W*H).  Per pixel: winner id
 * (0xFFFFFFFF for background), depth (float of s; +inf for background), rgb
 * (0 for background), the winner's smallest barycentric (edge distance;
 * +inf for background) and the relative depth gap to the next-nearest hit
 * of another triangle (+inf if there is none), and the smallest |min_k b_k|
 * over every other triangle whose plane the ray meets in front of the winner
 * (within a relative depth of 1e-3; any depth for background) -- the margin
 * by which no other triangle could take the pixel.  Any output may be NULL.
 */
void or_render(const or_view *v, int64_t V, int64_t T, const double *pos, const double *vel,
               const double *col, const int32_t *tri, const int64_t *pix, int64_t npix,
               uint32_t *id_out, float *depth_out, double *s_out, double *rgb_out, double *bmin_out,
               double *gap_out, double *near_out, double *cos_out)
{
    (void)V;
    /* camera-space start/end of every vertex, computed once */
    double *S = (double *)malloc(sizeof(double) * 3 * (V > 0 ? V : 1));
    double *E = (double *)malloc(sizeof(double) * 3 * (V > 0 ? V : 1));
    for (int64_t k = 0; k < V; ++k)
        vertex_start_end(v, pos, vel, k, S + 3 * k, E + 3 * k);

#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t n = 0; n < npix; ++n) {
        int64_t lin = pix ? pix[n] : n;
        int64_t i = lin % v->W, j = lin / v->W;
        double t, x[2], dir[3];
        or_pixel(v, i, j, &t, x, dir);

        int64_t best = -1;
        double best_s = INFINITY, second_s = INFINITY, best_b[3] = {0, 0, 0};
        for (int64_t id = 0; id < T; ++id) {
            double P[3][3], b[3], s;
            for (int k = 0; k < 3; ++k)
                lerp3(S + 3 * tri[3 * id + k], E + 3 * tri[3 * id + k], t, P[k]);
            int reg = cramer(P[0], P[1], P[2], dir, b, &s);
            if (!is_hit(reg, b, s, v->z_near))
                continue;
            if (s < best_s) { /* ids ascend, so equal s keeps the smaller id */
                second_s = best_s;
                best_s = s;
                best = id;
                memcpy(best_b, b, sizeof b);
            } else if (s < second_s) {
                second_s = s;
            }
        }
        if (id_out) id_out[n] = best < 0 ? 0xFFFFFFFFu : (uint32_t)best;
        if (depth_out) depth_out[n] = best < 0 ? INFINITY : (float)best_s;
        if (s_out) s_out[n] = best_s;
        if (bmin_out) {
            double m = best_b[0] < best_b[1] ? best_b[0] : best_b[1];
            bmin_out[n] = best < 0 ? INFINITY : (m < best_b[2] ? m : best_b[2]);
        }
        if (gap_out) gap_out[n] = best < 0 ? INFINITY : (second_s - best_s) / best_s;
        if (near_out) {
            /* second sweep: edge margin of every potential occluder */
            double m = INFINITY;
            for (int64_t id = 0; id < T; ++id) {
                if (id == best)
                    continue;
                double P[3][3], b[3], s;
                for (int k = 0; k < 3; ++k)
                    lerp3(S + 3 * tri[3 * id + k], E + 3 * tri[3 * id + k], t, P[k]);
                if (!cramer(P[0], P[1], P[2], dir, b, &s) || !(s > v->z_near))
                    continue;
                if (best >= 0 && s > best_s * (1.0 + 1e-3))
                    continue;
                double mb = b[0] < b[1] ? b[0] : b[1];
                mb = mb < b[2] ? mb : b[2];
                mb = fabs(mb);
                if (mb < m)
                    m = mb;
            }
            near_out[n] = m;
        }
        if (cos_out) {
            /* |cos| of the angle between the ray and the winner's plane
             * normal: the conditioning of its depth (1 for background) */
            double cg = 1.0;
            if (best >= 0) {
                double P[3][3], nh[3], len, flip;
                for (int k = 0; k < 3; ++k)
                    lerp3(S + 3 * tri[3 * best + k], E + 3 * tri[3 * best + k], t, P[k]);
                face_normal(P, dir, nh, &len, &flip);
                cg = fabs(dot(nh, dir)) / sqrt(dot(dir, dir));
            }
            cos_out[n] = cg;
        }
        if (rgb_out) {
            double rgb[3] = {0, 0, 0};
            if (best >= 0) {
                double P[3][3];
                for (int k = 0; k < 3; ++k)
                    lerp3(S + 3 * tri[3 * best + k], E + 3 * tri[3 * best + k], t, P[k]);
                shade(v, P, best_b, col, tri + 3 * best, t, dir, rgb);
            }
            for (int c = 0; c < 3; ++c)
                rgb_out[3 * n + c] = rgb[c];
        }
    }
    free(S);
    free(E);
}

/*
 * Evaluate one (pixel, triangle) pair without the inside test: out[0..2] =
 * barycentrics of the ray point in the plane, out[3] = ray parameter s,
 * out[4] = 1 if it counts as a hit, out[5] = distance (unit display
 * coordinates) from the pixel's display location to the boundary of the
 * triangle projected at the pixel time (0 if a vertex is not in front of
 * the camera).  Used to excuse GPU/oracle mismatches that sit on an edge or
 * a depth tie.
 */
void or_eval(const or_view *v, const double *pos, const double *vel, const int32_t *tri, int64_t lin,
             int64_t id, double out[6])
{
    int64_t i = lin % v->W, j = lin / v->W;
    double t, x[2], dir[3], P[3][3], b[3], s;
    or_pixel(v, i, j, &t, x, dir);
    tri_at(v, pos, vel, tri, id, t, P);
    int reg = cramer(P[0], P[1], P[2], dir, b, &s);
    out[0] = b[0];
    out[1] = b[1];
    out[2] = b[2];
    out[3] = s;
    out[4] = is_hit(reg, b, s, v->z_near);
    double q[3][2], dmin = INFINITY;
    int front = 1;
    for (int k = 0; k < 3; ++k) {
        if (!(P[k][2] > 0.0))
            front = 0;
        q[k][0] = (P[k][0] / (P[k][2] * v->tan_x) + 1.0) / 2.0;
        q[k][1] = (P[k][1] / (P[k][2] * v->tan_y) + 1.0) / 2.0;
    }
    for (int k = 0; k < 3 && front; ++k) {
        const double *a = q[k], *c = q[(k + 1) % 3];
        double e0 = c[0] - a[0], e1 = c[1] - a[1];
        double w0 = x[0] - a[0], w1 = x[1] - a[1];
        double ee = e0 * e0 + e1 * e1;
        double f = ee > 0.0 ? (w0 * e0 + w1 * e1) / ee : 0.0;
        f = f < 0.0 ? 0.0 : (f > 1.0 ? 1.0 : f);
        double d0 = w0 - f * e0, d1 = w1 - f * e1;
        double d = sqrt(d0 * d0 + d1 * d1);
        if (d < dmin)
            dmin = d;
    }
    out[5] = front ? dmin : 0.0;
}

/* ---------------------------------------------------------------- gradient */

/*
 * Gradient of sum_n sum_c g[n][c] * rgb[n][c] with respect to vertex colours,
 * positions and velocities, with the visible triangle of every pixel held
 * fixed (ids from the oracle's own render).  Chain: rgb = a sigma with
 * a = sum_k b_k col_k and sigma = k_a + k_d max(0, nhat . l); the
 * barycentrics of the ray point are b_k = w_k / (w_0 + w_1 + w_2) with
 * w_0 = dir.(B x C), w_1 = dir.(C x A), w_2 = dir.(A x B) (equal to the
 * Cramer solution); the moved vertex c(t) = (1-t)(R0 p + T0) + t(R1(p+v)+T1)
 * so dc/dp = (1-t) R0 + t R1 and dc/dv = t R1.  Outputs are accumulated
 * (+=) into dcol, dpos, dvel [V][3].
 */
void or_grad(const or_view *v, int64_t V, int64_t T, const double *pos, const double *vel,
             const double *col, const int32_t *tri, const int64_t *pix, int64_t npix,
             const uint32_t *ids, const double *g, double *dcol, double *dpos, double *dvel)
{
    (void)V;
    (void)T;
    for (int64_t n = 0; n < npix; ++n) {
        if (ids[n] == 0xFFFFFFFFu)
            continue;
        int64_t lin = pix ? pix[n] : n;
        int64_t i = lin % v->W, j = lin / v->W;
        int64_t id = ids[n];
        const int32_t *vid = tri + 3 * id;
        double t, x[2], dir[3], P[3][3], b[3], s;
        or_pixel(v, i, j, &t, x, dir);
        tri_at(v, pos, vel, tri, id, t, P);
        cramer(P[0], P[1], P[2], dir, b, &s);
        const double *A = P[0], *B = P[1], *C = P[2];
        const double *gn = g + 3 * n;

        double nh[3], len, flip, l[3];
        face_normal(P, dir, nh, &len, &flip);
        or_light(v, t, l);
        double ndl = dot(nh, l);
        double sigma = v->k_a + v->k_d * (ndl > 0.0 ? ndl : 0.0);

        /* colours */
        double a[3], gb[3];
        for (int c = 0; c < 3; ++c)
            a[c] = b[0] * col[3 * vid[0] + c] + b[1] * col[3 * vid[1] + c] + b[2] * col[3 * vid[2] + c];
        for (int k = 0; k < 3; ++k) {
            gb[k] = 0.0;
            for (int c = 0; c < 3; ++c) {
                dcol[3 * vid[k] + c] += gn[c] * b[k] * sigma;
                gb[k] += gn[c] * col[3 * vid[k] + c] * sigma;
            }
        }
        double gsig = gn[0] * a[0] + gn[1] * a[1] + gn[2] * a[2];

        /* barycentrics -> vertices */
        double w0, w1, w2, BxC[3], CxA[3], AxB[3];
        cross(B, C, BxC);
        cross(C, A, CxA);
        cross(A, B, AxB);
        w0 = dot(dir, BxC);
        w1 = dot(dir, CxA);
        w2 = dot(dir, AxB);
        double Ssum = w0 + w1 + w2;
        double bw0 = w0 / Ssum, bw1 = w1 / Ssum, bw2 = w2 / Ssum;
        double gdotb = gb[0] * bw0 + gb[1] * bw1 + gb[2] * bw2;
        double gw0 = (gb[0] - gdotb) / Ssum, gw1 = (gb[1] - gdotb) / Ssum, gw2 = (gb[2] - gdotb) / Ssum;
        double gA[3], gB[3], gC[3], tmp[3];
        double DxC[3], BxD[3], CxD[3], DxA[3], DxB[3], AxD[3];
        cross(dir, C, DxC);
        cross(B, dir, BxD);
        cross(C, dir, CxD);
        cross(dir, A, DxA);
        cross(dir, B, DxB);
        cross(A, dir, AxD);
        for (int r = 0; r < 3; ++r) {
            gA[r] = gw1 * DxC[r] + gw2 * BxD[r];
            gB[r] = gw0 * CxD[r] + gw2 * DxA[r];
            gC[r] = gw0 * DxB[r] + gw1 * AxD[r];
        }

        /* normal -> vertices: diffuse through n . l, specular through n . h */
        double hv[3] = {0.0, 0.0, 0.0}, ndh = 0.0;
        if (v->k_s > 0.0)
            ndh = half_vector(l, dir, nh, hv);
        const int spc = v->k_s > 0.0 && ndh > 0.0;
        if (ndl > 0.0 || spc) {
            const double gd = ndl > 0.0 ? gsig * v->k_d : 0.0;
            const double gs = spc ? (gn[0] + gn[1] + gn[2]) * v->k_s * v->shininess * pow(ndh, v->shininess - 1.0)
                                  : 0.0;
            double gnh[3] = {gd * l[0] + gs * hv[0], gd * l[1] + gs * hv[1], gd * l[2] + gs * hv[2]};
            double pr = dot(nh, gnh);
            double gnn[3];
            for (int r = 0; r < 3; ++r)
                gnn[r] = flip * (gnh[r] - pr * nh[r]) / len;
            double BmC[3] = {B[0] - C[0], B[1] - C[1], B[2] - C[2]};
            double CmA[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
            double AmB[3] = {A[0] - B[0], A[1] - B[1], A[2] - B[2]};
            cross(BmC, gnn, tmp);
            for (int r = 0; r < 3; ++r) gA[r] += tmp[r];
            cross(CmA, gnn, tmp);
            for (int r = 0; r < 3; ++r) gB[r] += tmp[r];
            cross(AmB, gnn, tmp);
            for (int r = 0; r < 3; ++r) gC[r] += tmp[r];
        }

        /* moved vertex -> position and velocity */
        const double *gv[3] = {gA, gB, gC};
        for (int k = 0; k < 3; ++k) {
            for (int c = 0; c < 3; ++c) {
                double dp = 0.0, dv = 0.0;
                for (int r = 0; r < 3; ++r) {
                    dp += ((1.0 - t) * v->pose0[4 * r + c] + t * v->pose1[4 * r + c]) * gv[k][r];
                    dv += t * v->pose1[4 * r + c] * gv[k][r];
                }
                dpos[3 * vid[k] + c] += dp;
                dvel[3 * vid[k] + c] += dv;
            }
        }
    }
}

/* Pixel times, display locations and ray directions for a pixel list. */
void or_pixels(const or_view *v, const int64_t *pix, int64_t npix, double *t_out, double *x_out,
               double *dir_out)
{
    for (int64_t n = 0; n < npix; ++n) {
        int64_t lin = pix ? pix[n] : n;
        or_pixel(v, lin % v->W, lin / v->W, t_out + n, x_out + 2 * n, dir_out + 3 * n);
    }
}

int or_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------- display unfoveation */

/* Sec. 3.1.1, "Display": the foveated framebuffer image I_f (planar rgb
 * [3][H][W]) is converted into the display image I_u (planar rgb
 * [3][Hd][Wd]) by I_u(x) = I_f(q^-1(x)).  Display pixel (a, b) has its
 * centre at x = ((a + 1/2)/Wd, (b + 1/2)/Hd); non-foveated views use the
 * identity map.  Two methods, as in the paper:
 *
 * method 0, MIP + cubic.  A MIP pyramid of I_f (level k + 1 = the average
 *   of each 2x2 block of level k, sizes ceil(W_k / 2) x ceil(H_k / 2),
 *   blocks cut by the border averaged over their texels, down to 1 x 1) is
 *   sampled tri-linearly: the level of detail is lambda = log2 of the
 *   largest stretch of q^-1 at x (radial p^-1' or tangential p^-1(r)/r)
 *   times max(W/Wd, H/Hd), clamped to the pyramid, and the two levels
 *   around it are blended by its fraction.  Within a level the texel
 *   coordinate s = u W_k - 1/2 is sampled with a 3-tap cubic filter: the
 *   nearest texel and its two neighbours per axis (clamped to the edge),
 *   weighted by the cubic B-spline at their distance from s and
 *   normalised by the weights' sum.
 *
 * method 1, projected 5 x 5.  The framebuffer pixel that holds u = q^-1(x)
 *   and its 5 x 5 neighbourhood are weighted by a Gaussian reconstruction
 *   filter r(d) = exp(-d^2 / (2 sigma^2)) of the display-space distance d
 *   (in display pixels) between x and q of each framebuffer pixel centre,
 *   normalised by the weights' sum (pixels outside the framebuffer are
 *   skipped).  The weights are taken relative to the nearest sample, whose
 *   factor cancels in the normalisation, so far from the framebuffer (where
 *   every sample is many display pixels away) they do not underflow.
 *
 * margin[k]: distance, in texels, of the discrete choices the result
 * depends on (the nearest texel of each level used, or the pixel that
 * holds u) from their decision boundaries; near zero, floating point
 * rounding may tip the choice.  pix: requested display pixels (b * Wd + a)
 * or NULL for all; out: [3][npix]. */

static double or_bspline3(double x)
{
    x = fabs(x);
    if (x < 1.0)
        return 2.0 / 3.0 - x * x + 0.5 * x * x * x;
    if (x < 2.0) {
        double y = 2.0 - x;
        return y * y * y / 6.0;
    }
    return 0.0;
}

int64_t or_mip_levels(int64_t W, int64_t H, int64_t *dims)
{
    int64_t L = 0;
    for (;;) {
        if (dims) {
            dims[2 * L] = W;
            dims[2 * L + 1] = H;
        }
        ++L;
        if (W == 1 && H == 1)
            return L;
        W = (W + 1) / 2;
        H = (H + 1) / 2;
    }
}

static double *or_mip_build(const float *rgb, int64_t W, int64_t H, int64_t *L_out, int64_t **dims_out,
                            int64_t **offs_out)
{
    int64_t L = or_mip_levels(W, H, NULL);
    int64_t *dims = malloc(sizeof(int64_t) * 2 * L), *offs = malloc(sizeof(int64_t) * (L + 1));
    or_mip_levels(W, H, dims);
    offs[0] = 0;
    for (int64_t k = 0; k < L; ++k)
        offs[k + 1] = offs[k] + 3 * dims[2 * k] * dims[2 * k + 1];
    double *pyr = malloc(sizeof(double) * offs[L]);
    for (int64_t i = 0; i < 3 * W * H; ++i)
        pyr[i] = (double)rgb[i];
    for (int64_t k = 1; k < L; ++k) {
        const int64_t w0 = dims[2 * k - 2], h0 = dims[2 * k - 1], w1 = dims[2 * k], h1 = dims[2 * k + 1];
        const double *src = pyr + offs[k - 1];
        double *dst = pyr + offs[k];
        for (int64_t c = 0; c < 3; ++c)
            for (int64_t y = 0; y < h1; ++y)
                for (int64_t x = 0; x < w1; ++x) {
                    double s = 0.0;
                    int n = 0;
                    for (int dy = 0; dy < 2; ++dy)
                        for (int dx = 0; dx < 2; ++dx) {
                            const int64_t sx = 2 * x + dx, sy = 2 * y + dy;
                            if (sx < w0 && sy < h0) {
                                s += src[c * w0 * h0 + sy * w0 + sx];
                                ++n;
                            }
                        }
                    dst[c * w1 * h1 + y * w1 + x] = s / n;
                }
    }
    *L_out = L;
    *dims_out = dims;
    *offs_out = offs;
    return pyr;
}

/* 3-tap cubic sample of one level at texel coordinates (s, t); returns the
 * margin of the nearest-texel choice. */
static double or_sample3(const double *lev, int64_t w, int64_t h, double s, double t, double out[3])
{
    const double fs = floor(s + 0.5), ft = floor(t + 0.5);
    /* the nearest texel flips where s (or t) crosses n + 1/2 */
    const double margin = fmin(0.5 - fabs(s - fs), 0.5 - fabs(t - ft));
    double wx[3], wy[3], sx = 0.0, sy = 0.0;
    for (int k = 0; k < 3; ++k) {
        wx[k] = or_bspline3(s - (fs + k - 1));
        wy[k] = or_bspline3(t - (ft + k - 1));
        sx += wx[k];
        sy += wy[k];
    }
    out[0] = out[1] = out[2] = 0.0;
    for (int ky = 0; ky < 3; ++ky)
        for (int kx = 0; kx < 3; ++kx) {
            int64_t x = (int64_t)fs + kx - 1, y = (int64_t)ft + ky - 1;
            x = x < 0 ? 0 : (x >= w ? w - 1 : x);
            y = y < 0 ? 0 : (y >= h ? h - 1 : y);
            const double wgt = wx[kx] * wy[ky] / (sx * sy);
            for (int c = 0; c < 3; ++c)
                out[c] += wgt * lev[c * w * h + y * w + x];
        }
    return margin;
}

/* Unclamped level of detail of method 0 at display location x. */
double or_unfoveate_lod(const or_view *v, const double x[2], int64_t Wd, int64_t Hd)
{
    const int fov = v->mode == OR_FOVEATED || v->mode == OR_BOTH;
    double stretch = 1.0;
    if (fov) {
        const double e0 = x[0] - v->fovea[0], e1 = x[1] - v->fovea[1], r = sqrt(e0 * e0 + e1 * e1);
        if (v->p_n > 0) {
            stretch = r > 0.0 ? fmax(lut_pinv(v, r) / r, lut_dpinv(v, r)) : lut_dpinv(v, 0.0);
        } else {
            const double tang = r > 0.0 ? pow(r / OR_D, 1.0 / v->alpha - 1.0) : INFINITY;
            stretch = fmax(tang, tang / v->alpha);
        }
    }
    return log2(stretch * fmax((double)v->W / (double)Wd, (double)v->H / (double)Hd));
}

void or_unfoveate(const or_view *v, const float *rgb, int64_t Wd, int64_t Hd, int32_t method, double sigma,
                  const int64_t *pix, int64_t npix, double *out, double *margin)
{
    const int64_t W = v->W, H = v->H;
    const int fov = v->mode == OR_FOVEATED || v->mode == OR_BOTH;
    int64_t L = 0, *dims = NULL, *offs = NULL;
    double *pyr = method == 0 ? or_mip_build(rgb, W, H, &L, &dims, &offs) : NULL;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < npix; ++k) {
        const int64_t lin = pix ? pix[k] : k;
        const int64_t a = lin % Wd, b = lin / Wd;
        const double x[2] = {((double)a + 0.5) / (double)Wd, ((double)b + 0.5) / (double)Hd};
        double u[2];
        if (fov)
            or_qinv(v, x, u);
        else {
            u[0] = x[0];
            u[1] = x[1];
        }
        double res[3] = {0.0, 0.0, 0.0}, mg = INFINITY;
        if (method == 0) {
            /* largest stretch of q^-1 at x: radial d p^-1/dr = (1/alpha)(r/D)^(1/alpha - 1),
             * tangential p^-1(r)/r = (r/D)^(1/alpha - 1) */
            double lambda = or_unfoveate_lod(v, x, Wd, Hd);
            if (!(lambda > 0.0))
                lambda = 0.0;
            if (lambda > (double)(L - 1))
                lambda = (double)(L - 1);
            const int64_t k0 = (int64_t)floor(lambda), k1 = k0 + 1 < L ? k0 + 1 : k0;
            const double f = lambda - (double)k0;
            double s0[3], s1[3];
            const int64_t w0 = dims[2 * k0], h0 = dims[2 * k0 + 1], w1 = dims[2 * k1], h1 = dims[2 * k1 + 1];
            mg = or_sample3(pyr + offs[k0], w0, h0, u[0] * w0 - 0.5, u[1] * h0 - 0.5, s0);
            const double m1 = or_sample3(pyr + offs[k1], w1, h1, u[0] * w1 - 0.5, u[1] * h1 - 0.5, s1);
            if (f > 0.0)
                mg = fmin(mg, m1);
            for (int c = 0; c < 3; ++c)
                res[c] = (1.0 - f) * s0[c] + f * s1[c];
        } else {
            const double su = u[0] * (double)W, sv = u[1] * (double)H;
            const double fi = floor(su), fj = floor(sv);
            mg = fmin(fmin(su - fi, 1.0 - (su - fi)), fmin(sv - fj, 1.0 - (sv - fj)));
            int64_t i = (int64_t)fi, j = (int64_t)fj;
            i = i < 0 ? 0 : (i >= W ? W - 1 : i);
            j = j < 0 ? 0 : (j >= H ? H - 1 : j);
            /* squared display distances of the window's pixels (NAN: outside) */
            double d2[25], d2min = INFINITY;
            for (int dy = -2; dy <= 2; ++dy)
                for (int dx = -2; dx <= 2; ++dx) {
                    const int64_t pi = i + dx, pj = j + dy;
                    double *slot = &d2[(dy + 2) * 5 + dx + 2];
                    *slot = NAN;
                    if (pi < 0 || pj < 0 || pi >= W || pj >= H)
                        continue;
                    const double c_u[2] = {((double)pi + 0.5) / (double)W, ((double)pj + 0.5) / (double)H};
                    double c_x[2];
                    if (fov)
                        or_q(v, c_u, c_x);
                    else {
                        c_x[0] = c_u[0];
                        c_x[1] = c_u[1];
                    }
                    const double d0 = (x[0] - c_x[0]) * (double)Wd, d1 = (x[1] - c_x[1]) * (double)Hd;
                    *slot = d0 * d0 + d1 * d1;
                    d2min = fmin(d2min, *slot);
                }
            /* weights relative to the nearest sample: the common factor
             * exp(-d2min / (2 sigma^2)) cancels in the normalisation */
            double wsum = 0.0;
            for (int dy = -2; dy <= 2; ++dy)
                for (int dx = -2; dx <= 2; ++dx) {
                    const double q2 = d2[(dy + 2) * 5 + dx + 2];
                    if (isnan(q2))
                        continue;
                    const double wgt = exp(-(q2 - d2min) / (2.0 * sigma * sigma));
                    wsum += wgt;
                    for (int c = 0; c < 3; ++c)
                        res[c] += wgt * (double)rgb[c * W * H + (j + dy) * W + (i + dx)];
                }
            for (int c = 0; c < 3; ++c)
                res[c] /= wsum;
        }
        for (int c = 0; c < 3; ++c)
            out[c * npix + k] = res[c];
        if (margin)
            margin[k] = mg;
    }
    free(pyr);
    free(dims);
    free(offs);
}
