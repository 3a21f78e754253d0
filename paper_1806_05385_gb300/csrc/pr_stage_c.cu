// pr_stage_c.cu -- stage (c): per-fragment ray casting (Sec. 3.2,
// "Intersection") inside the tile bins of stage (b), and the resolve of the
// packed depth|id keys into the id and depth buffers.
//
// Work decomposition: a persistent grid pulls (view, tile, bin run) items
// from a global atomic queue.  One CTA covers one S x S tile; each warp owns
// an 8 x 8 pixel block and each lane two pixels of one column (rows r and
// r + 4), so under a horizontal rolling scan both pixels share one time.
// The bin run of an item comes sorted by nearest depth (stage b).  Every
// warp walks it on its own, 32 entries at a time: the lanes screen the
// entries against the block (depth cut, display box, time interval) while
// the records stream into the warp's shared memory, then the warp runs the
// watertight test for the survivors, each lane for its two pixels.  Per
// pixel the nearest key is kept in a register and merged into the frame
// with one 64-bit atomicMin per item.
#include "pr_launch.h"

namespace pr {

// Error allowances of the precision form.  kRelCoord bounds the error of
// an FP32 sheared vertex coordinate relative to the coordinate magnitudes
// it was computed from (camera-space transform, interpolation to the pixel
// time, shear, and the foveation power of the ray: a few ulps each, with a
// safety factor of about 3); kTieRel is the relative depth difference under
// which two hits count as tied.
constexpr float kRelCoord = 2e-6f;
constexpr float kTieRel = 1e-4f;
constexpr float kKeySlack = 1e-3f;
// A winning hit whose FP32 depth may be off by more than kDepthRel
// (relative) also goes to the FP64 re-test, which writes the FP64 depth
// rounded to FP32.  kRelCoordDepth is the error of a sheared FP32
// coordinate relative to the magnitudes it came from that this estimate
// assumes: about 3 ulps (the transform, the interpolation to the pixel
// time and the shear round once or twice each), not the worst-case
// allowance kRelCoord of the inside/outside decision.
constexpr float kDepthRel = 8e-6f;
constexpr float kRelCoordDepth = 2e-7f;

// One watertight ray/triangle test (Woop, Benthin and Wald, "Watertight
// Ray/Triangle Intersection", JCGT 2013) of the ray from the origin along
// (dx, dy, 1) against the triangle moved to time t.  With dz = 1 the
// shear/scale constants are Sx = dx, Sy = dy, Sz = 1.  The edge-function
// products are rounded separately (no contraction) so that a shared edge
// yields exactly opposite values in its two triangles; zero counts as
// either sign (inclusive edges).
//
// A hit's depth is T / det.  Its key only matters if it can beat the
// pixel's current best, so the exact depth (IEEE division) is computed only
// when T / det <= best_depth (1 + 2^-20), tested as a product; the margin
// keeps every candidate that could win or tie, so the result is the exact
// minimum key whatever the order of the triangles.
//
// kFlag (precision form): also decide whether FP32 settles this pair.  The
// edge functions carry an error of at most e (from the allowance on the
// sheared coordinates); a pair whose inside/outside outcome is not certain
// within e, or a hit that ties the current best within kTieRel, sets `flag`
// when it could still decide the pixel (its plane lies in front of the best
// hit, within the tie allowance).  kDepthFlag (the fragment stage's
// precision form): a hit that becomes the pixel's best also sets `flag` when
// its depth is ill-conditioned.  Moving sheared vertex k by at most c_k per
// coordinate moves the plane's depth on the ray (the z axis) by at most
// (sum_k b_k c_k) (1 + (|Nx| + |Ny|) / |Nz|) to first order, with b_k the
// hit's barycentrics, N the normal of the sheared triangle and |Nz| =
// |det|: a grazing ray has a large tangent.  c_k is kRelCoordDepth times
// the magnitude vertex k's coordinates came from.
template <bool kFlag, bool kDepthFlag = false>
__device__ __forceinline__ void ray_test(const float4 r0, const float4 r1, const float4 r2, const float4 r3,
                                         const float d2y, const float d2z, const float t, const float dx,
                                         const float dy, const float zn, const uint32_t id, unsigned long long &best,
                                         float &best_depth, unsigned &hits, bool &flag)
{
    // vertices at time t (c = S + t D), sheared so the ray is the z axis
    const float Az = fmaf(t, r2.w, r0.z), Bz = fmaf(t, r3.z, r1.y), Cz = fmaf(t, d2z, r2.x);
    const float ax = fmaf(-dx, Az, fmaf(t, r2.y, r0.x)), ay = fmaf(-dy, Az, fmaf(t, r2.z, r0.y));
    const float bx = fmaf(-dx, Bz, fmaf(t, r3.x, r0.w)), by = fmaf(-dy, Bz, fmaf(t, r3.y, r1.x));
    const float cx = fmaf(-dx, Cz, fmaf(t, r3.w, r1.z)), cy = fmaf(-dy, Cz, fmaf(t, d2y, r1.w));
    const float U = __fsub_rn(__fmul_rn(cx, by), __fmul_rn(cy, bx));
    const float V = __fsub_rn(__fmul_rn(ax, cy), __fmul_rn(ay, cx));
    const float W = __fsub_rn(__fmul_rn(bx, ay), __fmul_rn(by, ax));
    const bool outside = fminf(U, fminf(V, W)) < 0.f && fmaxf(U, fmaxf(V, W)) > 0.f;
    if (!kFlag) {
        if (outside)
            return;
    }
    const float det = U + V + W;
    const float T = fmaf(U, Az, fmaf(V, Bz, W * Cz));
    const float adet = fabsf(det), aT = det < 0.f ? -T : T;  // depth = aT / adet
    if (kFlag) {
        const float sm = fmaxf(fabsf(ax) + fabsf(ay), fmaxf(fabsf(bx) + fabsf(by), fabsf(cx) + fabsf(cy)));
        const float zm = fmaxf(fabsf(Az), fmaxf(fabsf(Bz), fabsf(Cz)));
        const float ec = kRelCoord * (zm * (1.f + fabsf(dx) + fabsf(dy)) + sm);
        const float e = 2.f * ec * (sm + ec) + 1e-30f;
        const bool sure_in = (U > e && V > e && W > e) || (U < -e && V < -e && W < -e);
        const bool sure_out = (U > e || V > e || W > e) && (U < -e || V < -e || W < -e);
        if (!sure_in && !sure_out &&
            (!(adet > 0.f) || (aT > zn * (1.f - kTieRel) * adet && aT <= best_depth * (1.f + kTieRel) * adet)))
            flag = true;
        if (outside)
            return;
    }
    if (!(adet > 0.f) || !(aT > zn * adet))
        return;
    ++hits;
    if (kFlag && aT >= best_depth * (1.f - kTieRel) * adet && aT <= best_depth * (1.f + kTieRel) * adet)
        flag = true;
    if (aT > best_depth * 1.00000095f * adet)
        return;  // behind the current best: cannot win
    const float depth = __fdiv_rn(T, det);
    if (!(depth > zn))
        return;
    const unsigned long long key = pack_key(depth, id);
    if (key < best) {
        best = key;
        best_depth = depth;
        if (kFlag && kDepthFlag) {
            const float e1x = bx - ax, e1y = by - ay, e1z = Bz - Az, e2x = cx - ax, e2y = cy - ay, e2z = Cz - Az;
            const float nx = fabsf(fmaf(e1y, e2z, -e1z * e2y)), ny = fabsf(fmaf(e1z, e2x, -e1x * e2z));
            const float sd = 1.f + fabsf(dx) + fabsf(dy);
            // sum_k b_k |coordinates of k| times |det| (U, V, W share det's sign on a hit)
            const float magb = fabsf(U) * fmaf(fabsf(Az), sd, fabsf(ax) + fabsf(ay)) +
                               fabsf(V) * fmaf(fabsf(Bz), sd, fabsf(bx) + fabsf(by)) +
                               fabsf(W) * fmaf(fabsf(Cz), sd, fabsf(cx) + fabsf(cy));
            if (kRelCoordDepth * magb * (adet + nx + ny) > kDepthRel * depth * adet * adet)
                flag = true;
        }
    }
}

// Build-time knob of the fragment kernel: the occupancy it is compiled for
// (resident warps per SM, which caps registers).
#ifndef PR_FRAG_WARPS
#define PR_FRAG_WARPS 24
#endif
#define PR_FRAG_MINB(nt) (PR_FRAG_WARPS > 0 ? (PR_FRAG_WARPS * 32) / (nt) : 1)

// Marks pixel g for the FP64 re-test (once: a bitmap de-duplicates the
// pixels that several items flag) and appends it to the flag list.
__device__ __forceinline__ void flag_pixel(long long g, unsigned *flag_bits, long long *flag_list, Counters *cnt)
{
    const unsigned bit = 1u << (g & 31);
    if (!(atomicOr(&flag_bits[g >> 5], bit) & bit)) {
        const unsigned long long k = atomicAdd(&cnt->flagged, 1ull);
        flag_list[k] = g;
    }
}

// Order-preserving int image of a float (and back), for warp min/max
// reductions of float values with the integer redux instruction.
__device__ __forceinline__ int fkey(float f)
{
    const int i = __float_as_int(f);
    return i ^ ((i >> 31) & 0x7FFFFFFF);
}
__device__ __forceinline__ float funkey(int i) { return __int_as_float(i ^ ((i >> 31) & 0x7FFFFFFF)); }
__device__ __forceinline__ float warp_minf(float x) { return funkey(__reduce_min_sync(0xffffffffu, fkey(x))); }
__device__ __forceinline__ float warp_maxf(float x) { return funkey(__reduce_max_sync(0xffffffffu, fkey(x))); }

// 16-byte asynchronous global -> shared copy (L1-cached), and the wait for
// all of this thread's copies.
__device__ __forceinline__ void copy16_async(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void copy_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Records staged per warp and triangle: S and D of the three vertices
// (float4 0-3 of the record) and the time interval / D2yz float4 (5).
constexpr int kStageF4 = 5;

template <int S, bool kFlag>
__global__ void __launch_bounds__(S *S / 2, PR_FRAG_MINB(S *S / 2))
    k_fragment(const ViewDev *__restrict__ views, const int4 *__restrict__ items,
               const unsigned long long *__restrict__ scan, long long tile_lo, long long tile_hi, long long cap_items,
               int *__restrict__ head, const unsigned long long *__restrict__ pairs, const float4 *__restrict__ rec,
               unsigned long long *__restrict__ keys, unsigned *__restrict__ flag_bits,
               long long *__restrict__ flag_list, Counters *cnt)
{
    constexpr int NT = S * S / 2;  // threads: two pixels each
    constexpr int NW = NT / 32;    // warps
    constexpr int WPR = S / 8;     // 8x8 warp blocks per tile row
    __shared__ float4 s_rec[NW][32 * kStageF4];  // per warp: the records of its current 32 candidates
    __shared__ long long s_item[2];

    // an attempt whose bins overflowed is rerun by the host: entries of the
    // dropped hits were never written, so nothing here may read the bins;
    // the same after a scan that gave up its wait (the frame is an error)
    if (cnt->status & (ST_OVERFLOW_PAIRS | ST_OVERFLOW_ITEMS | ST_TIMEOUT))
        return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ci = (warp % WPR) * 8 + (lane & 7);
    const int cj0 = (warp / WPR) * 8 + (lane >> 3), cj1 = cj0 + 4;
    const long long it_lo = (long long)(scan[tile_lo] >> 40);
    const long long it_hi = min((long long)(scan[tile_hi] >> 40), cap_items);
    float4 *wrec = s_rec[warp];
    unsigned long long n_tests = 0, n_hits = 0;

    if (threadIdx.x == 0)
        s_item[0] = it_lo + atomicAdd(head, 1);
    __syncthreads();
    for (int par = 0;; par ^= 1) {
        const long long it = s_item[par];
        if (it >= it_hi)
            break;
        if (threadIdx.x == 0)  // the next item, fetched while this one runs
            s_item[par ^ 1] = it_lo + atomicAdd(head, 1);
        const int4 item = items[it];
        const ViewDev &v = views[item.x];
        const int tx = item.y % v.tiles_x, ty = item.y / v.tiles_x;
        const int i = tx * S + ci, j0 = ty * S + cj0, j1 = ty * S + cj1;
        const bool ok0 = i < v.W && j0 < v.H, ok1 = i < v.W && j1 < v.H;
        float x00, x01, t0, dx0, dy0, x10, x11, t1, dx1, dy1;
        pixel_ray(v, min(i, v.W - 1), min(j0, v.H - 1), x00, x01, t0, dx0, dy0);
        pixel_ray(v, min(i, v.W - 1), min(j1, v.H - 1), x10, x11, t1, dx1, dy1);
        // the warp's block in display space and time (valid pixels only)
        const float wx0 = warp_minf(fminf(ok0 ? x00 : INFINITY, ok1 ? x10 : INFINITY));
        const float wx1 = warp_maxf(fmaxf(ok0 ? x00 : -INFINITY, ok1 ? x10 : -INFINITY));
        const float wy0 = warp_minf(fminf(ok0 ? x01 : INFINITY, ok1 ? x11 : INFINITY));
        const float wy1 = warp_maxf(fmaxf(ok0 ? x01 : -INFINITY, ok1 ? x11 : -INFINITY));
        // with a horizontal scan (d1 = 0) the time strip is already part of
        // every triangle's display box; otherwise test the interval too
        float wt0 = -INFINITY, wt1 = INFINITY;
        if (is_rolling(v.mode) && v.d1 != 0.f) {
            wt0 = warp_minf(fminf(ok0 ? t0 : INFINITY, ok1 ? t1 : INFINITY));
            wt1 = warp_maxf(fmaxf(ok0 ? t0 : -INFINITY, ok1 ? t1 : -INFINITY));
        }
        const float zn = v.z_near;
        const unsigned id_base = (unsigned)v.tri_off;
        unsigned long long best0 = ~0ull, best1 = ~0ull;
        float bd0 = INFINITY, bd1 = INFINITY;
        unsigned hits = 0, tested = 0;
        bool fl0 = false, fl1 = false;
        // The run is sorted nearest first (stage b).  Once a triangle cannot
        // come nearer than every pixel's current best (with a margin for the
        // FP32 depth; for the precision form also the tie band), no later
        // one can change a pixel of this warp.  The lanes screen 32 entries
        // at a time (depth cut, display box, time interval) while their
        // records stream into the warp's shared memory; the warp then runs
        // the ray tests for the survivors, in order.
        const float cull = kFlag ? (1.f + 3.f * kTieRel) : 1.f;
        for (int k0 = item.z; k0 < item.w; k0 += 32) {
            float wmax = warp_maxf(fmaxf(ok0 ? bd0 : 0.f, ok1 ? bd1 : 0.f)) * cull;
            const int kk = k0 + lane;
            const unsigned long long e = kk < item.w ? pairs[kk] : ~0ull;
            const float key = depth_from_order_key((unsigned)(e >> 32));
            const unsigned stopm = __ballot_sync(0xffffffffu, kk >= item.w || key * 0.99999f > wmax);
            // entries ascend, so every lane from the first stop on stops too
            const int ncand = stopm ? __ffs(stopm) - 1 : 32;
            const unsigned gid = (unsigned)e;
            float d2y = 0.f, d2z = 0.f;
            bool take = false;
            if (lane < ncand) {
                const float4 *r = rec + (size_t)gid * kRecF4;
#pragma unroll
                for (int f = 0; f < 4; ++f)
                    copy16_async(wrec + lane * kStageF4 + f, r + f);
                const float4 bb = __ldg(r + 4), tb = __ldg(r + 5);
                d2y = tb.z;
                d2z = tb.w;
                take = !(bb.x > wx1 || bb.y < wx0 || bb.z > wy1 || bb.w < wy0 || tb.x > wt1 || tb.y < wt0);
            }
            copy_async_wait_all();
            __syncwarp();
            unsigned live = __ballot_sync(0xffffffffu, take);
            bool stop = stopm != 0u;
            while (live) {
                const int k = __ffs(live) - 1;
                live &= live - 1u;
                // the bests move with every test: re-check the cut before each
                // (every 8 tests instead: 0.098 ms against 0.089 on the HMD
                // frame, 0.385 against 0.276 ms on the 1M-triangle frame)
                wmax = warp_maxf(fmaxf(ok0 ? bd0 : 0.f, ok1 ? bd1 : 0.f)) * cull;
                if (__shfl_sync(0xffffffffu, key, k) * 0.99999f > wmax) {
                    stop = true;
                    break;
                }
                const float4 r0 = wrec[k * kStageF4 + 0], r1 = wrec[k * kStageF4 + 1];
                const float4 r2 = wrec[k * kStageF4 + 2], r3 = wrec[k * kStageF4 + 3];
                const float ky = __shfl_sync(0xffffffffu, d2y, k), kz = __shfl_sync(0xffffffffu, d2z, k);
                const unsigned id = __shfl_sync(0xffffffffu, gid, k) - id_base;
                ++tested;
                ray_test<kFlag, kFlag>(r0, r1, r2, r3, ky, kz, t0, dx0, dy0, zn, id, best0, bd0, hits, fl0);
                ray_test<kFlag, kFlag>(r0, r1, r2, r3, ky, kz, t1, dx1, dy1, zn, id, best1, bd1, hits, fl1);
            }
            if (stop)
                break;
            __syncwarp();  // the staged records are no longer read
        }
        n_tests += (unsigned long long)tested * (unsigned)(ok0 + ok1);
        n_hits += hits;
        const long long g0 = v.pix_off + (long long)j0 * v.W + i, g1 = v.pix_off + (long long)j1 * v.W + i;
        if (ok0 && best0 != ~0ull)
            atomicMin(&keys[g0], best0);
        if (ok1 && best1 != ~0ull)
            atomicMin(&keys[g1], best1);
        if (kFlag) {
            if (ok0 && fl0)
                flag_pixel(g0, flag_bits, flag_list, cnt);
            if (ok1 && fl1)
                flag_pixel(g1, flag_bits, flag_list, cnt);
        }
        __syncthreads();  // s_item[par ^ 1] is written; s_item[par] may be reused
    }
    for (int o = 16; o > 0; o >>= 1) {
        n_tests += __shfl_xor_sync(0xffffffffu, n_tests, o);
        n_hits += __shfl_xor_sync(0xffffffffu, n_hits, o);
    }
    // one pair of global atomics per CTA (every thread left the loop at the
    // same item)
    __shared__ unsigned long long s_tests, s_hits;
    if (threadIdx.x == 0)
        s_tests = s_hits = 0ull;
    __syncthreads();
    if (lane == 0) {
        atomicAdd(&s_tests, n_tests);
        atomicAdd(&s_hits, n_hits);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(&cnt->tests, s_tests);
        atomicAdd(&cnt->hits, s_hits);
    }
}

template <int S, bool kFlag>
static int grid_for()
{
    static int g = 0;
    if (g == 0) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fragment<S, kFlag>, S * S / 2, 0);
        g = sms * (per > 0 ? per : 1);
    }
    return g;
}

int fragment_grid(int S, bool flag)
{
    if (flag)
        return S == 8 ? grid_for<8, true>() : (S == 16 ? grid_for<16, true>() : grid_for<32, true>());
    return S == 8 ? grid_for<8, false>() : (S == 16 ? grid_for<16, false>() : grid_for<32, false>());
}

template <bool kFlag>
static cudaError_t launch_fragment_t(int S, const ViewDev *views, const int4 *items, const unsigned long long *scan,
                                     long long tile_lo, long long tile_hi, long long cap_items, int *head,
                                     const unsigned long long *pairs, const float4 *rec, unsigned long long *keys,
                                     unsigned *flag_bits, long long *flag_list, Counters *cnt, int grid,
                                     cudaStream_t st)
{
    switch (S) {
    case 8:
        k_fragment<8, kFlag><<<grid, 32, 0, st>>>(views, items, scan, tile_lo, tile_hi, cap_items, head, pairs,
                                                  rec, keys, flag_bits, flag_list, cnt);
        break;
    case 16:
        k_fragment<16, kFlag><<<grid, 128, 0, st>>>(views, items, scan, tile_lo, tile_hi, cap_items, head,
                                                    pairs, rec, keys, flag_bits, flag_list, cnt);
        break;
    case 32:
        k_fragment<32, kFlag><<<grid, 512, 0, st>>>(views, items, scan, tile_lo, tile_hi, cap_items, head,
                                                    pairs, rec, keys, flag_bits, flag_list, cnt);
        break;
    default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t launch_fragment(int S, bool flag, const ViewDev *views, const int4 *items, const unsigned long long *scan,
                            long long tile_lo, long long tile_hi, long long cap_items, int *head,
                            const unsigned long long *pairs, const float4 *rec, unsigned long long *keys,
                            unsigned *flag_bits, long long *flag_list, Counters *cnt, int grid, cudaStream_t st)
{
    if (flag)
        return launch_fragment_t<true>(S, views, items, scan, tile_lo, tile_hi, cap_items, head, pairs, rec,
                                       keys, flag_bits, flag_list, cnt, grid, st);
    return launch_fragment_t<false>(S, views, items, scan, tile_lo, tile_hi, cap_items, head, pairs, rec, keys,
                                    flag_bits, flag_list, cnt, grid, st);
}

// ---------------------------------------------------------------- FP64 re-test

// The map from a vertex (p, v) to its sheared camera-space position at the
// pixel's time, in FP64: with M = (1-t) R0 + t R1, N = t R1 and
// T = (1-t) T0 + t T1 the moved vertex is c = M p + N v + T (the same
// point as (1-t)(R0 p + T0) + t(R1 (p + v) + T1)), and the shear of the
// watertight test takes rows x - dx z, y - dy z, z.  Built once per pixel,
// it leaves 18 multiply-adds per vertex.
struct Shear64 {
    double P[3][3], Q[3][3], c[3];
};

__device__ Shear64 shear64(const ViewDev &v, const Ray64 &ry)
{
    Shear64 sh;
    double M[3][3], N[3][3], T[3];
    for (int r = 0; r < 3; ++r) {
        for (int k = 0; k < 3; ++k) {
            M[r][k] = (1.0 - ry.t) * (double)v.R0[3 * r + k] + ry.t * (double)v.R1[3 * r + k];
            N[r][k] = ry.t * (double)v.R1[3 * r + k];
        }
        T[r] = (1.0 - ry.t) * (double)v.T0[r] + ry.t * (double)v.T1[r];
    }
    const double d[2] = {ry.dx, ry.dy};
    for (int k = 0; k < 3; ++k) {
        for (int r = 0; r < 2; ++r) {
            sh.P[r][k] = M[r][k] - d[r] * M[2][k];
            sh.Q[r][k] = N[r][k] - d[r] * N[2][k];
        }
        sh.P[2][k] = M[2][k];
        sh.Q[2][k] = N[2][k];
    }
    for (int r = 0; r < 2; ++r)
        sh.c[r] = T[r] - d[r] * T[2];
    sh.c[2] = T[2];
    return sh;
}

__device__ __forceinline__ double3 sheared64(const ViewDev &v, const Shear64 &sh, int k)
{
    const float4 va = v.vtx[2 * k], vb = v.vtx[2 * k + 1];
    const double p[3] = {va.x, va.y, va.z};
    const double w[3] = {va.w, vb.x, vb.y};
    double a[3];
    for (int r = 0; r < 3; ++r)
        a[r] = sh.c[r] + sh.P[r][0] * p[0] + sh.P[r][1] * p[1] + sh.P[r][2] * p[2] + sh.Q[r][0] * w[0] +
               sh.Q[r][1] * w[1] + sh.Q[r][2] * w[2];
    return make_double3(a[0], a[1], a[2]);
}

// Watertight test in FP64; on a hit beyond the near plane returns true with
// the ray parameter as the fraction num / den, den > 0 (the division is left
// to the caller, who needs it only for the winner).
__device__ bool hit64(const ViewDev &v, const Shear64 &sh, int tri, double &num, double &den)
{
    const int4 tv = v.tri4[tri];
    const double3 A = sheared64(v, sh, tv.x), B = sheared64(v, sh, tv.y), C = sheared64(v, sh, tv.z);
    const double ax = A.x, ay = A.y, bx = B.x, by = B.y, cx = C.x, cy = C.y;
    const double U = cx * by - cy * bx, V = ax * cy - ay * cx, W = bx * ay - by * ax;
    if ((U < 0.0 || V < 0.0 || W < 0.0) && (U > 0.0 || V > 0.0 || W > 0.0))
        return false;
    const double det = U + V + W;
    if (det == 0.0)
        return false;
    const double T = U * A.z + V * B.z + W * C.z;
    num = det < 0.0 ? -T : T;
    den = fabs(det);
    return num > (double)v.z_near * den;
}

// Each warp re-decides up to 32 flagged pixels.  Sweep 1 runs the FP32
// test with the error allowance over the pixel's whole tile bin and finds
// the nearest hit that FP32 settles ("robust").  Sweep 2 re-evaluates in
// FP64 every pair that could still beat it: unsettled pairs whose plane
// lies in front of it and hits tied with it.  Every other pair is a settled
// miss or a settled hit behind it, so the FP64 minimum over the candidates
// is the exact winner.
//
// The FP32 sweeps of one pixel run across the warp's lanes (one bin entry
// each), the pixels one after the other; their FP64 candidates go to a
// per-warp list in shared memory, grouped by pixel.  FP64 runs at a small
// fraction of the FP32 rate on this part, so the FP64 tests then run with
// one lane per pixel, in step across the warp: each FP64 instruction serves
// up to 32 pixels instead of one candidate.  Candidates that do not fit the
// list are tested at once and kept as the pixel's running best.
//
// A bin entry carries a lower bound of the nearest depth its triangle
// reaches (the depth order key, rounded down); a pair whose bound lies
// behind the sweep's current limit by more than kKeySlack cannot be nearer
// (an unsettled pair's plane point lies within the edge allowance, about
// 1e-5 relative, of the triangle), so both sweeps skip its test.
constexpr int kRetestWarps = 4;
constexpr int kRetestList = 512;  // candidates listed per warp and round of 32 pixels

// An FP64 hit kept as the fraction num / den (den > 0; den = 0: none) with
// its triangle; `better` orders by depth, then by the smaller id.
struct Hit64 {
    double num, den;
    unsigned id;
};

__device__ __forceinline__ bool better(double num, double den, unsigned id, const Hit64 &b)
{
    if (b.den == 0.0)
        return true;
    const double l = num * b.den, r = b.num * den;  // num / den vs b.num / b.den
    return l < r || (l == r && id < b.id);
}

// The pixel of flag f: its view, column, row, and its tile bin [off, off + n).
struct RetestPixel {
    const ViewDev *v;
    long long g, off, n;
    int i, j;
};

__device__ __forceinline__ RetestPixel retest_pixel(const ViewDev *views, int nviews, const long long *pix_offs,
                                                    const unsigned long long *scan,
                                                    const unsigned long long *tile_cnt, const long long *flag_list,
                                                    long long f, long long cap_pairs)
{
    RetestPixel px;
    px.g = flag_list[f];
    px.v = &views[find_view(pix_offs, nviews, px.g)];
    const ViewDev &v = *px.v;
    const long long lin = px.g - v.pix_off;
    px.j = (int)lin / v.W;  // lin < 2^28
    px.i = (int)lin - px.j * v.W;
    const long long tile = v.tile_off + (long long)(px.j / v.S) * v.tiles_x + px.i / v.S;
    px.off = (long long)(scan[tile] & 0xFFFFFFFFFFull);
    px.n = min((long long)(tile_cnt[tile] & 0xFFFFFFFFFFull), max(cap_pairs - px.off, 0ll));
    return px;
}

__global__ void __launch_bounds__(kRetestWarps * 32) k_retest(const ViewDev *__restrict__ views, int nviews,
                                                              const long long *__restrict__ pix_offs,
                                                              const unsigned long long *__restrict__ scan,
                                                              const unsigned long long *__restrict__ tile_cnt,
                                                              const unsigned long long *__restrict__ pairs,
                                                              const float4 *__restrict__ rec,
                                                              const long long *__restrict__ flag_list,
                                                              unsigned long long *__restrict__ keys, long long cap_pairs,
                                                              Counters *cnt)
{
    // an attempt whose bins overflowed is rerun by the host; its bin counts
    // reach past the entries that were written (a scan timeout: the same)
    if (cnt->status & (ST_OVERFLOW_PAIRS | ST_OVERFLOW_ITEMS | ST_OVERFLOW_FLAGS | ST_TIMEOUT))
        return;
    __shared__ unsigned s_list[kRetestWarps][kRetestList];  // candidate triangles, grouped by pixel
    __shared__ int s_start[kRetestWarps][32], s_count[kRetestWarps][32];
    __shared__ Hit64 s_best[kRetestWarps][32];  // per pixel: the best of the candidates tested at once
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long nflag = (long long)cnt->flagged;
    const long long nw = (long long)gridDim.x * kRetestWarps;
    // pixels per warp and round: spread over every warp of the grid (the
    // pixels of a warp run one after the other), at most 32
    const long long per = max(1ll, min(32ll, (nflag + nw - 1) / nw));
    for (long long f0 = ((long long)blockIdx.x * kRetestWarps + w) * per; f0 < nflag; f0 += nw * per) {
        const int npx = (int)min(per, nflag - f0);
        int used = 0;  // list entries in use (the same in every lane)
        for (int q = 0; q < npx; ++q) {
            const RetestPixel px = retest_pixel(views, nviews, pix_offs, scan, tile_cnt, flag_list, f0 + q, cap_pairs);
            const ViewDev &v = *px.v;
            float x0, x1, t, dx, dy;
            pixel_ray(v, px.i, px.j, x0, x1, t, dx, dy);
            const float zn = v.z_near;
            const unsigned id_base = (unsigned)v.tri_off;
            // sweep 1: nearest settled hit (each lane a share of the bin)
            float rb = INFINITY;
            for (long long k = lane; k < px.n; k += 32) {
                const unsigned long long ent = pairs[px.off + k];
                if (depth_from_order_key((unsigned)(ent >> 32)) > rb * (1.f + kKeySlack))
                    continue;  // behind this lane's nearest settled hit
                const unsigned gid = (unsigned)ent;
                const float4 *r = rec + (size_t)gid * kRecF4;
                unsigned long long best = ~0ull;
                float bd = INFINITY;
                unsigned hits = 0;
                bool fl = false;
                ray_test<true>(r[0], r[1], r[2], r[3], r[5].z, r[5].w, t, dx, dy, zn, gid - id_base, best, bd, hits,
                               fl);
                if (best != ~0ull && !fl)
                    rb = fminf(rb, bd);
            }
            rb = warp_minf(rb);
            // sweep 2: list the pairs that could beat it
            const float lim = rb * (1.f + 2.f * kTieRel);
            const int start = used;
            Hit64 ib{0.0, 0.0, 0xFFFFFFFFu};
            for (long long k0 = 0; k0 < px.n; k0 += 32) {
                const long long k = k0 + lane;
                bool cand = false;
                unsigned id = 0u;
                if (k < px.n) {
                    const unsigned long long ent = pairs[px.off + k];
                    if (depth_from_order_key((unsigned)(ent >> 32)) <= lim * (1.f + kKeySlack)) {
                        const unsigned gid = (unsigned)ent;
                        const float4 *r = rec + (size_t)gid * kRecF4;
                        unsigned long long best = ~0ull;
                        float bd = lim;  // "best so far" = the limit, so fl marks pairs in front of it
                        unsigned hits = 0;
                        bool fl = false;
                        ray_test<true>(r[0], r[1], r[2], r[3], r[5].z, r[5].w, t, dx, dy, zn, gid - id_base, best, bd,
                                       hits, fl);
                        cand = fl || best != ~0ull;  // not a settled miss, nor a settled hit behind the limit
                        id = gid - id_base;
                    }
                }
                const unsigned m = __ballot_sync(0xffffffffu, cand);
                if (!m)
                    continue;
                if (used + __popc(m) <= kRetestList) {
                    if (cand)
                        s_list[w][used + __popc(m & ((1u << lane) - 1u))] = id;
                    used += __popc(m);
                } else if (cand) {  // the list is full: test now
                    const Shear64 sh = shear64(v, pixel_ray64(v, px.i, px.j));
                    double num, den;
                    if (hit64(v, sh, (int)id, num, den) && better(num, den, id, ib))
                        ib = Hit64{num, den, id};
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double on = __shfl_xor_sync(0xffffffffu, ib.num, o);
                const double od = __shfl_xor_sync(0xffffffffu, ib.den, o);
                const unsigned oi = __shfl_xor_sync(0xffffffffu, ib.id, o);
                if (od > 0.0 && better(on, od, oi, ib))
                    ib = Hit64{on, od, oi};
            }
            if (lane == 0) {
                s_start[w][q] = start;
                s_count[w][q] = used - start;
                s_best[w][q] = ib;
            }
        }
        __syncwarp();
        // the listed candidates in FP64, one lane per pixel
        if (lane < npx) {
            const RetestPixel px = retest_pixel(views, nviews, pix_offs, scan, tile_cnt, flag_list, f0 + lane,
                                                cap_pairs);
            const ViewDev &v = *px.v;
            Hit64 b = s_best[w][lane];
            const int c0 = s_start[w][lane], c1 = c0 + s_count[w][lane];
            if (c1 > c0) {
                const Shear64 sh = shear64(v, pixel_ray64(v, px.i, px.j));
                for (int c = c0; c < c1; ++c) {
                    const unsigned id = s_list[w][c];
                    double num, den;
                    if (hit64(v, sh, (int)id, num, den) && better(num, den, id, b))
                        b = Hit64{num, den, id};
                }
            }
            const unsigned bid = b.den > 0.0 ? b.id : 0xFFFFFFFFu;
            const double bs = b.den > 0.0 ? b.num / b.den : 0.0;
            const unsigned long long key = bid == 0xFFFFFFFFu ? ~0ull : pack_key((float)bs, bid);
            const unsigned long long old = keys[px.g];
            if (old != ~0ull && bid != 0xFFFFFFFFu && (unsigned)(old & 0xFFFFFFFFull) == bid) {
                // same winner: record the FP32 depth error against FP64
                const double d32 = (double)__uint_as_float((unsigned)(old >> 32));
                const float rel = (float)(fabs(d32 - bs) / bs);
                atomicMax(&cnt->depth_err_bits, __float_as_uint(rel));
            }
            if (old != key) {
                keys[px.g] = key;
                atomicAdd(&cnt->changed, 1ull);
            }
        }
        __syncwarp();  // the list is reused by the next round
    }
}

int retest_grid()
{
    static int g = 0;
    if (g == 0) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        g = sms * 8;
    }
    return g;
}

cudaError_t launch_retest(const ViewDev *views, int nviews, const long long *pix_offs, const unsigned long long *scan,
                          const unsigned long long *tile_cnt, const unsigned long long *pairs, const float4 *rec,
                          const long long *flag_list, unsigned long long *keys, long long cap_pairs, Counters *cnt,
                          cudaStream_t st)
{
    k_retest<<<retest_grid(), kRetestWarps * 32, 0, st>>>(views, nviews, pix_offs, scan, tile_cnt, pairs, rec,
                                                          flag_list, keys, cap_pairs, cnt);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- resolve

__global__ void k_resolve(const ViewDev *__restrict__ views, int nviews, const long long *__restrict__ pix_offs,
                          long long npix, unsigned long long *__restrict__ keys, int reset_keys)
{
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= npix)
        return;
    const ViewDev &v = views[find_view(pix_offs, nviews, g)];
    const long long lin = g - v.pix_off;
    const unsigned long long key = keys[g];
    const bool bg = key == ~0ull;
    if (!bg && reset_keys)
        keys[g] = ~0ull;  // left as the next frame wants it
    if (v.id_out)
        v.id_out[lin] = bg ? 0xFFFFFFFFu : (unsigned)(key & 0xFFFFFFFFull);
    if (v.depth_out)
        v.depth_out[lin] = bg ? INFINITY : __uint_as_float((unsigned)(key >> 32));
}

cudaError_t launch_resolve(const ViewDev *views, int nviews, const long long *pix_offs, long long npix,
                           unsigned long long *keys, bool reset_keys, cudaStream_t st)
{
    if (npix > 0)
        k_resolve<<<(unsigned)((npix + 255) / 256), 256, 0, st>>>(views, nviews, pix_offs, npix, keys, reset_keys);
    return cudaGetLastError();
}

}  // namespace pr
