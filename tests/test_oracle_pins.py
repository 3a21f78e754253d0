"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: an
independent pinhole rasterizer (the classic special case), exact rational
arithmetic, closed-form motion under a rolling scan, hand-computed shading,
finite differences, and the invariants of the foveation map.  A plausible
slip in the oracle (a dropped term, a swapped index, a transposed pose, the
wrong lerp weight, the wrong time axis) fails at least one of them.
"""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

from paper_1806_05385_gb300 import scenes as S

BG = 0xFFFFFFFF


def _f32(x):
    return float(np.float32(x))


def mkview(W=16, H=12, mode=S.MODE_CLASSIC, tan=(0.5, 0.5), pose0=None, pose1=None, fovea=(0.5, 0.5),
           alpha=2.0, d=(1.0, 0.0), light=(0.0, 0.0, -1.0), k_a=0.1, k_d=0.9, k_s=0.0, shininess=1.0):
    """A view whose parameters are FP32 values (the method's inputs are the
    FP32 values of the library's ABI; the oracle widens them exactly), so the
    independent computations below see exactly what the oracle sees."""
    I = np.eye(4, dtype=np.float32)
    return S.View(W=W, H=H, tan_x=_f32(tan[0]), tan_y=_f32(tan[1]), pose0=I if pose0 is None else pose0,
                  pose1=(I if pose0 is None else pose0) if pose1 is None else pose1, mode=mode,
                  fovea=(_f32(fovea[0]), _f32(fovea[1])), alpha=_f32(alpha), d=(_f32(d[0]), _f32(d[1])),
                  light_w=tuple(_f32(x) for x in light), k_a=_f32(k_a), k_d=_f32(k_d), k_s=_f32(k_s),
                  shininess=_f32(shininess))


# --------------------------------------------------------------------------
# foveation map q (Sec. 3.1.1)
# --------------------------------------------------------------------------

def test_warp_fixed_point_inverse_radial(oracle):
    rng = np.random.default_rng(1)
    for _ in range(200):
        f = rng.uniform(0.05, 0.95, 2).astype(np.float32).astype(np.float64)
        v = mkview(fovea=tuple(f), alpha=float(rng.uniform(1.0, 4.0)))
        assert np.array_equal(oracle.q(v, f), f)            # the fovea is a fixed point
        x = rng.uniform(0, 1, 2)
        assert np.allclose(oracle.q(v, oracle.qinv(v, x)), x, atol=1e-12, rtol=0)
        u = rng.uniform(0, 1, 2)
        assert np.allclose(oracle.qinv(v, oracle.q(v, u)), u, atol=1e-12, rtol=0)
        a, b = u - f, oracle.q(v, u) - f                     # radial lines are kept
        assert abs(a[0] * b[1] - a[1] * b[0]) < 1e-12 and a @ b > 0
        assert np.linalg.norm(b) <= np.linalg.norm(a) + 1e-15  # p(d) <= d on (0, sqrt 2)


def test_warp_identity_and_domain_end(oracle):
    rng = np.random.default_rng(2)
    v1 = mkview(fovea=(0.3, 0.6), alpha=1.0)                # constant density: classic
    for _ in range(20):
        u = rng.uniform(0, 1, 2)
        assert np.allclose(oracle.q(v1, u), u, atol=1e-15)
    v = mkview(fovea=(0.0, 0.0), alpha=2.0)                 # p(sqrt 2) = sqrt 2
    assert np.allclose(oracle.q(v, np.array([1.0, 1.0])), [1.0, 1.0], atol=1e-15)
    assert oracle.p(math.sqrt(2.0), 3.0) == pytest.approx(math.sqrt(2.0), abs=1e-15)
    assert oracle.p(0.5, 1.0) == pytest.approx(0.5, abs=1e-16)


def test_warp_density_magnifies_fovea(oracle):
    """Framebuffer pixels per display area (det of the Jacobian of q^-1)
    falls with the distance r from the fovea: magnified (> 1) near it and
    compressed (< 1) in the far periphery (Sec. 3.1.1).  For the radial map
    det = p^-1(r) p^-1'(r) / r, with p^-1(r) = D (r/D)^(1/alpha):
    det = (1/alpha) (r/D)^(2/alpha - 2), which is 1 at r = D alpha^(alpha/(2-2 alpha))."""
    D = math.sqrt(2.0)
    for alpha in (1.5, 2.0, 3.0):
        v = mkview(fovea=(0.05, 0.05), alpha=alpha)

        def jdet(x, h=1e-7):
            J = np.zeros((2, 2))
            for k in range(2):
                e = np.zeros(2)
                e[k] = h
                J[:, k] = (oracle.qinv(v, x + e) - oracle.qinv(v, x - e)) / (2 * h)
            return np.linalg.det(J)

        dets = []
        for r in (0.01, 0.1, 0.3, 0.6, 0.9, 1.2):
            x = np.array([0.05, 0.05]) + r * np.array([0.6, 0.8])
            dets.append(jdet(x))
            assert dets[-1] == pytest.approx((1.0 / alpha) * (r / D) ** (2.0 / alpha - 2.0), rel=1e-5)
        assert all(a > b for a, b in zip(dets, dets[1:]))
        assert dets[0] > 1.0 and dets[-1] < 1.0


# --------------------------------------------------------------------------
# pixel time and ray (Sec. 3.1.2, conventions)
# --------------------------------------------------------------------------

def test_pixel_time_rolling_scans_columns(oracle):
    W, H = 7, 5
    t, x, d = oracle.pixels(mkview(W=W, H=H, mode=S.MODE_ROLLING))
    t = t.reshape(H, W)
    assert np.all(t == t[0:1, :])                           # one time per column (d = (1,0))
    assert np.all(np.diff(t[0]) > 0) and 0 < t.min() and t.max() < 1
    assert t[0, 0] == pytest.approx(0.5 / W) and t[0, -1] == pytest.approx(1 - 0.5 / W)
    for mode in (S.MODE_CLASSIC, S.MODE_FOVEATED):
        assert np.all(oracle.pixels(mkview(W=W, H=H, mode=mode))[0] == 0)
    # joint mode: time of a pixel = rolling time of its display location q(u)
    vb = mkview(W=W, H=H, mode=S.MODE_BOTH, fovea=(0.3, 0.7))
    tb, xb, _ = oracle.pixels(vb)
    lin = np.arange(W * H)
    u = np.stack([(lin % W + 0.5) / W, (lin // W + 0.5) / H], 1)
    xq = np.array([oracle.q(vb, uu) for uu in u])
    assert np.allclose(xb, xq, atol=0) and np.allclose(tb, xq[:, 0], atol=0)
    # a scan along y with a 10 % blank period (Sec. 3.1.2, d = (0, .9))
    ty = oracle.pixels(mkview(W=W, H=H, mode=S.MODE_ROLLING, d=(0.0, 0.9)))[0].reshape(H, W)
    assert np.all(ty == ty[:, 0:1]) and ty.max() < 0.9


def test_centre_ray_is_optical_axis(oracle):
    W, H = 5, 3
    _, x, d = oracle.pixels(mkview(W=W, H=H, tan=(0.7, 0.3)))
    c = 1 * W + 2
    assert np.allclose(d[c], [0, 0, 1], atol=0)
    # top-left pixel looks left and up (x right, y down)
    assert d[0, 0] < 0 and d[0, 1] < 0
    assert d[0, 0] == pytest.approx((2 * 0.5 / W - 1) * 0.7)


def _q_closed_form(u, f, alpha):
    """q(u) = f + (u - f)/|u - f| * D (|u - f|/D)^alpha, D = sqrt 2, written
    out here on its own (Sec. 3.1.1 with the power p of Sec. 5.1)."""
    D = math.sqrt(2.0)
    e = np.asarray(u, dtype=np.float64) - f
    r = math.hypot(e[0], e[1])
    return f.copy() if r == 0.0 else f + e * (D * (r / D) ** alpha / r)


@pytest.mark.parametrize("mode", [S.MODE_FOVEATED, S.MODE_BOTH])
def test_foveated_ray_goes_through_the_display_location(oracle, mode):
    """Sec. 3.1.1: a foveated pixel u is seen along the ray of its display
    location q(u), dir = ((2 q0 - 1) tanX, (2 q1 - 1) tanY, 1); the joint
    mode takes the same ray (Sec. 3.1.3).  The fovea is off centre and
    alpha = 2, so the ray of u itself differs from it by up to a few tenths
    and this tells dir(q(u)) from dir(u)."""
    W, H = 9, 7
    v = mkview(W=W, H=H, mode=mode, tan=(0.7, 0.4), fovea=(0.3, 0.65), alpha=2.0)
    _, x, d = oracle.pixels(v)
    f = np.array(v.fovea, dtype=np.float64)
    worst_u = 0.0
    for k in range(W * H):
        u = np.array([(k % W + 0.5) / W, (k // W + 0.5) / H])
        xq = _q_closed_form(u, f, 2.0)
        want = np.array([(2 * xq[0] - 1) * v.tan_x, (2 * xq[1] - 1) * v.tan_y, 1.0])
        assert np.allclose(x[k], xq, rtol=0, atol=1e-14)
        assert np.allclose(d[k], want, rtol=0, atol=1e-14)
        du = np.array([(2 * u[0] - 1) * v.tan_x, (2 * u[1] - 1) * v.tan_y, 1.0])
        worst_u = max(worst_u, float(np.abs(du - want).max()))
    assert worst_u > 0.1


def _seg_dist_sampled(p, a, b, n=20001):
    """Distance from p to the segment ab by brute force over n points."""
    s = np.linspace(0.0, 1.0, n)[:, None]
    pts = a[None, :] * (1 - s) + b[None, :] * s
    return float(np.sqrt(((pts - p[None, :]) ** 2).sum(1)).min())


def _right_triangle_boundary_distance(p, a0, b0, a1, b1):
    """Distance from an interior point p to the boundary of the right
    triangle (a0, b0), (a1, b0), (a0, b1): the smallest of its distances to
    the two legs and to the hypotenuse line."""
    w, h = a1 - a0, b1 - b0
    hyp = abs((p[0] - a0) * h + (p[1] - b0) * w - w * h) / math.hypot(w, h)
    return min(p[0] - a0, p[1] - b0, hyp)


@pytest.mark.parametrize("mode,vx", [(S.MODE_CLASSIC, 0.0), (S.MODE_ROLLING, 0.4), (S.MODE_BOTH, 0.4)])
def test_eval_display_edge_distance_closed_form(oracle, mode, vx):
    """or_eval's sixth output, the distance in unit display coordinates from
    a pixel's display location to the boundary of the triangle projected at
    the pixel time (it decides which FP32 id mismatches are excused).  A
    fronto-parallel triangle at depth z whose display image is the right
    triangle (a0, b0), (a1, b0), (a0, b1), translating along camera x by a
    display distance V per frame: at the pixel time t its image is shifted by
    V t (Sec. 3.1.2).  Inside: the smallest distance to the legs and the
    hypotenuse line; everywhere: brute force over points of the three
    edges.  The display location is q(u) in the joint mode (Sec. 3.1.1)."""
    W, H, z, tx, ty = 24, 20, 4.0, 0.5, 0.375   # tangents exact in FP32
    a0, b0, a1, b1 = 0.25, 0.3, 0.8, 0.9
    disp = np.array([[a0, b0], [a1, b0], [a0, b1]])
    cam = np.stack([(2 * disp[:, 0] - 1) * tx * z, (2 * disp[:, 1] - 1) * ty * z, np.full(3, z)], 1)
    vel = np.zeros((3, 3))
    vel[:, 0] = vx * 2 * tx * z            # camera x displacement that moves the image by vx
    tri = np.array([[0, 1, 2]], dtype=np.int32)
    v = mkview(W=W, H=H, mode=mode, tan=(tx, ty), fovea=(0.55, 0.45))
    f = np.array(v.fovea, dtype=np.float64)
    checked_inside = 0
    for k in range(W * H):
        u = np.array([(k % W + 0.5) / W, (k // W + 0.5) / H])
        x = _q_closed_form(u, f, 2.0) if mode == S.MODE_BOTH else u
        t = x[0] if mode != S.MODE_CLASSIC else 0.0
        sh = np.array([vx * t, 0.0])
        A, B, C = disp[0] + sh, disp[1] + sh, disp[2] + sh
        ev = oracle.evaluate(v, cam, vel, tri, k, 0)
        want = min(_seg_dist_sampled(x, A, B), _seg_dist_sampled(x, B, C), _seg_dist_sampled(x, C, A))
        assert ev[5] == pytest.approx(want, abs=5e-5)   # sampling error <= edge length / 40000
        xs = x - sh
        inside = xs[0] >= a0 and xs[1] >= b0 and (xs[0] - a0) / (a1 - a0) + (xs[1] - b0) / (b1 - b0) <= 1
        assert bool(ev[4]) == inside
        if inside:
            checked_inside += 1
            assert ev[5] == pytest.approx(_right_triangle_boundary_distance(xs, a0, b0, a1, b1), abs=1e-12)
    assert checked_inside > 40
    # a vertex behind the camera: no projected triangle, distance 0
    cam2 = cam.copy()
    cam2[0, 2] = -1.0
    assert oracle.evaluate(v, cam2, vel, tri, (H // 2) * W + W // 2, 0)[5] == 0.0


@pytest.mark.parametrize("g,h", [(0.5, 0.0), (0.0, -0.8), (1.3, 0.6)])
def test_depth_conditioning_cosine_of_a_tilted_plane(oracle, g, h):
    """The oracle's `cos` output, |cos| of the angle between a pixel's ray
    and its winner's plane normal (it sets the depth allowance of the parity
    rule), against a hand-computed normal: the plane z = 5 + g x + h y has
    the normal (-g, -h, 1), so cos = |d . (-g, -h, 1)| / (|d| sqrt(1 + g^2 +
    h^2)) for the pixel ray d."""
    W, H, tx, ty = 12, 10, 0.5, 0.5
    plane = lambda X, Y: 5.0 + g * X + h * Y
    corners = [(-4.0, -4.0), (4.0, -4.0), (0.0, 4.0)]
    pos = np.array([[X, Y, plane(X, Y)] for X, Y in corners])
    v = mkview(W=W, H=H, tan=(tx, ty))
    o = oracle.render(v, pos, np.zeros_like(pos), np.ones_like(pos), np.array([[0, 1, 2]], np.int32))
    hit = o["id"] == 0
    assert hit.sum() > W * H // 3
    n = np.array([-g, -h, 1.0]) / math.sqrt(1 + g * g + h * h)
    for k in np.nonzero(hit)[0]:
        d = np.array([(2 * ((k % W) + 0.5) / W - 1) * tx, (2 * ((k // W) + 0.5) / H - 1) * ty, 1.0])
        assert o["cos"][k] == pytest.approx(abs(d @ n) / np.linalg.norm(d), rel=1e-12)
    assert np.all(o["cos"][~hit] == 1.0)


# --------------------------------------------------------------------------
# classic special case == an independent pinhole rasterizer
# --------------------------------------------------------------------------

def pinhole_raster(view, pos, tri):
    """Independent FP64 rasterizer for a static scene at t = 0: project the
    vertices, 2D edge functions at pixel centres (inclusive), perspective
    correct depth by interpolating 1/z in the image plane, nearest wins."""
    M = np.asarray(view.pose0, dtype=np.float64)
    P = pos.astype(np.float64) @ M[:3, :3].T + M[:3, 3]
    s = P[:, :2] / P[:, 2:3]
    W, H = view.W, view.H
    jj, ii = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    px = (2 * (ii + 0.5) / W - 1) * view.tan_x
    py = (2 * (jj + 0.5) / H - 1) * view.tan_y
    best = np.full((H, W), np.inf)
    bid = np.full((H, W), BG, dtype=np.uint64)
    margin = np.full((H, W), np.inf)
    depths = []
    for k, (a, b, c) in enumerate(tri):
        def edge(p0, p1):
            return (p1[0] - p0[0]) * (py - p0[1]) - (p1[1] - p0[1]) * (px - p0[0])
        e0, e1, e2 = edge(s[b], s[c]), edge(s[c], s[a]), edge(s[a], s[b])
        area = e0 + e1 + e2
        l0, l1, l2 = e0 / area, e1 / area, e2 / area
        inside = (l0 >= 0) & (l1 >= 0) & (l2 >= 0)
        z = 1.0 / (l0 / P[a, 2] + l1 / P[b, 2] + l2 / P[c, 2])
        margin = np.minimum(margin, np.abs(np.minimum(np.minimum(l0, l1), l2)))
        z = np.where(inside, z, np.inf)
        depths.append(z)
        upd = z < best
        best = np.where(upd, z, best)
        bid = np.where(upd, k, bid)
    depths = np.sort(np.stack(depths), axis=0)
    with np.errstate(invalid="ignore"):
        gap = (depths[1] - depths[0]) / depths[0] if len(tri) > 1 else np.full((H, W), np.inf)
    return bid.astype(np.uint32).ravel(), best.ravel(), margin.ravel(), np.nan_to_num(gap, nan=np.inf).ravel()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_classic_equals_pinhole_raster(oracle, seed):
    rng = np.random.default_rng(seed)
    T = 20
    pos = rng.uniform([-1, -1, 2], [1, 1, 6], size=(3 * T, 3)).astype(np.float32)
    tri = np.arange(3 * T, dtype=np.int32).reshape(T, 3)
    R = S.rot_pitch(7.0) @ S.rot_yaw(-11.0)
    pose = S.make_pose(R, (0.1, -0.2, 0.3))                 # a static, non-trivial pose
    v = mkview(W=24, H=18, tan=(0.6, 0.45), pose0=pose)
    zero = np.zeros_like(pos)
    o = oracle.render(v, pos, zero, np.ones_like(pos), tri)
    rid, rz, margin, gap = pinhole_raster(v, pos, tri)
    ok = (margin > 1e-9) & (gap > 1e-12)
    assert ok.mean() > 0.95
    assert np.array_equal(o["id"][ok], rid[ok])
    hit = ok & (rid != BG)
    assert hit.sum() > 50
    assert np.allclose(o["s"][hit], rz[hit], rtol=1e-12, atol=0)


def test_pose_translation_shifts_image(oracle):
    """World->camera pose: translating the world by +x moves the image right."""
    pos = np.array([[-0.2, -0.2, 4.0], [0.2, -0.2, 4.0], [0.0, 0.3, 4.0]], dtype=np.float32)
    tri = np.array([[0, 1, 2]], dtype=np.int32)
    z = np.zeros_like(pos)
    cols = []
    for tx in (0.0, 0.5):
        v = mkview(W=40, H=20, pose0=S.make_pose(np.eye(3), (tx, 0.0, 0.0)))
        ids = oracle.render(v, pos, z, z, tri)["id"].reshape(20, 40)
        cols.append(np.nonzero((ids != BG).any(0))[0].mean())
    # 0.5 units at depth 4 with tan 0.5 is 0.5/4/0.5/2 * 40 = 5 pixels
    assert cols[1] - cols[0] == pytest.approx(5.0, abs=0.6)


# --------------------------------------------------------------------------
# exact rational arithmetic on tiny inputs (moving, rolling, posed)
# --------------------------------------------------------------------------

def _exact_eval(view, pos, vel, tri, lin, k):
    W, H = view.W, view.H
    i, j = lin % W, lin // W
    u0, u1 = Fr(2 * i + 1, 2 * W), Fr(2 * j + 1, 2 * H)
    t = u0 * Fr(view.d[0]) + u1 * Fr(view.d[1])
    dx = (2 * u0 - 1) * Fr(view.tan_x)
    dy = (2 * u1 - 1) * Fr(view.tan_y)
    D = (dx, dy, Fr(1))
    M0 = [[Fr(float(x)) for x in row] for row in np.asarray(view.pose0, np.float64)]
    M1 = [[Fr(float(x)) for x in row] for row in np.asarray(view.pose1, np.float64)]
    V = []
    for vi in tri[k]:
        p = [Fr(float(x)) for x in pos[vi]]
        pe = [p[r] + Fr(float(vel[vi][r])) for r in range(3)]
        s0 = [sum(M0[r][c] * p[c] for c in range(3)) + M0[r][3] for r in range(3)]
        s1 = [sum(M1[r][c] * pe[c] for c in range(3)) + M1[r][3] for r in range(3)]
        V.append([(1 - t) * s0[r] + t * s1[r] for r in range(3)])

    def cross(a, b):
        return (a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0])

    def dot(a, b):
        return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]

    A, B, Cc = V
    w = [dot(D, cross(B, Cc)), dot(D, cross(Cc, A)), dot(D, cross(A, B))]
    tot = sum(w)
    if tot == 0:
        return None
    b = [x / tot for x in w]
    s = dot(A, cross(B, Cc)) / tot
    return b, s


def test_exact_rational_bruteforce(oracle):
    rng = np.random.default_rng(7)
    T = 6
    pos = rng.uniform([-0.5, -0.5, 2], [0.5, 0.5, 4], size=(3 * T, 3)).astype(np.float32)
    vel = rng.normal(0, 0.1, size=(3 * T, 3)).astype(np.float32)
    tri = np.arange(3 * T, dtype=np.int32).reshape(T, 3)
    pose0 = S.make_pose(S.rot_yaw(3.0), (0.05, 0.0, 0.1))
    pose1 = S.make_pose(S.rot_pitch(2.0) @ S.rot_yaw(-4.0), (0.0, 0.02, -0.1))
    v = mkview(W=10, H=8, mode=S.MODE_ROLLING, pose0=pose0, pose1=pose1, tan=(0.25, 0.25))
    checked = 0
    for lin in range(0, 80):
        for k in range(T):
            ex = _exact_eval(v, pos, vel, tri, lin, k)
            ob = oracle.evaluate(v, pos, vel, tri, lin, k)
            if ex is None:
                continue
            b, s = ex
            assert np.allclose(ob[:3], [float(x) for x in b], rtol=1e-9, atol=1e-12)
            assert ob[3] == pytest.approx(float(s), rel=1e-12)
            if min(abs(x) for x in b) > 1e-12:
                exact_hit = all(x > 0 for x in b) and s > Fr(v.z_near)
                assert bool(ob[4]) == exact_hit
                checked += exact_hit
    assert checked > 5


# --------------------------------------------------------------------------
# rolling scan, closed forms (Sec. 3.1.2, Sec. 4.2.4)
# --------------------------------------------------------------------------

def _inside2d(tri2, p):
    (ax, ay), (bx, by), (cx, cy) = tri2
    px, py = p

    def e(x0, y0, x1, y1):
        return (x1 - x0) * (py - y0) - (y1 - y0) * (px - x0)

    e0, e1, e2 = e(bx, by, cx, cy), e(cx, cy, ax, ay), e(ax, ay, bx, by)
    area = e0 + e1 + e2
    lam = np.stack([e0 / area, e1 / area, e2 / area])
    return lam.min(0)


@pytest.mark.parametrize("vx", [0.3, -0.25])
def test_rolling_mover_closed_form(oracle, vx):
    """Fronto-parallel triangle at depth z moving along x at vx per frame,
    static camera, scan t = x: the scan catches a point at screen speed V
    (unit/frame) when x0 + V t = t (the linear Zenon case), so the rolling
    image is the still image sampled at ((1 - V) x, y)."""
    z, tan = 4.0, 0.5
    W, H = 97, 61
    pos = np.array([[-0.6, -0.5, z], [0.5, -0.3, z], [-0.1, 0.6, z]], dtype=np.float32)
    vel = np.tile(np.array([[vx, 0.0, 0.0]], dtype=np.float32), (3, 1))
    tri = np.array([[0, 1, 2]], dtype=np.int32)
    v = mkview(W=W, H=H, mode=S.MODE_ROLLING, tan=(tan, tan))
    o = oracle.render(v, pos, vel, np.ones_like(pos), tri)
    V = vx / (2.0 * z * tan)
    tri2 = [((p[0] / z / tan + 1) / 2, (p[1] / z / tan + 1) / 2) for p in pos.astype(np.float64)]
    jj, ii = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    xu, yu = (ii.ravel() + 0.5) / W, (jj.ravel() + 0.5) / H
    lam = _inside2d(tri2, ((1 - V) * xu, yu))
    ok = np.abs(lam) > 1e-9
    pred = lam >= 0
    assert np.array_equal((o["id"] != BG)[ok], pred[ok])
    assert pred.sum() > 100
    assert np.allclose(o["s"][pred & ok], z, rtol=1e-12)


def test_rolling_camera_yaw_catch_up(oracle):
    """A still point ahead of a camera that yaws during scan-out appears at
    the column where the scan catches its camera-space path (found here by
    bisection on the interpolated start/end camera positions)."""
    W, H, tan = 400, 9, 0.5
    yaw = 10.0
    R1 = S.rot_yaw(yaw)
    p = np.array([0.0, 0.0, 5.0])
    h = 0.03
    pos = np.array([p + [-h, -h, 0], p + [h, -h, 0], p + [0, h, 0]], dtype=np.float32)
    tri = np.array([[0, 1, 2]], dtype=np.int32)
    v = mkview(W=W, H=H, mode=S.MODE_ROLLING, tan=(tan, tan), pose1=S.make_pose(R1))
    ids = oracle.render(v, pos, np.zeros_like(pos), np.ones_like(pos), tri)["id"].reshape(H, W)
    cols = np.nonzero((ids != BG).any(0))[0]

    def xu(t):
        c = (1 - t) * p + t * (R1 @ p)
        return (c[0] / c[2] / tan + 1) / 2

    lo, hi = 0.0, 1.0
    for _ in range(80):
        mid = (lo + hi) / 2
        if xu(mid) > mid:
            lo = mid
        else:
            hi = mid
    col = lo * W - 0.5
    assert lo > 0.5                                          # +yaw turns the camera so the point drifts right
    assert cols.size > 0 and abs(cols.mean() - col) < 1.5


# --------------------------------------------------------------------------
# shading (Sec. 3.2 "Shading")
# --------------------------------------------------------------------------

def _flat(z=5.0, c=(0.2, 0.5, 0.8)):
    pos = np.array([[-3, -3, z], [3, -3, z], [0, 3, z]], dtype=np.float32)
    col = np.tile(np.array([c], dtype=np.float32), (3, 1))
    return pos, col, np.array([[0, 1, 2]], dtype=np.int32)


@pytest.mark.parametrize("light,sigma", [((0, 0, -1), 1.0), ((1, 0, 0), 0.1), ((0, 0, 1), 0.1),
                                         ((math.sin(math.pi / 3), 0, -0.5), 0.1 + 0.9 * 0.5)])
def test_shading_flat_closed_form(oracle, light, sigma):
    pos, col, tri = _flat()
    v = mkview(W=9, H=9, light=light)
    o = oracle.render(v, pos, np.zeros_like(pos), col, tri)
    c = 4 * 9 + 4
    assert o["id"][c] == 0
    assert np.allclose(o["rgb"][c], np.array([0.2, 0.5, 0.8]) * sigma, atol=1e-15)


def test_shading_barycentric_albedo(oracle):
    """Vertex colours red/green/blue on a fronto-parallel triangle facing the
    light: rgb equals the image-plane barycentrics (constant depth)."""
    z = 5.0
    pos = np.array([[-2.0, -2.0, z], [2.0, -1.0, z], [-0.5, 2.0, z]], dtype=np.float32)
    col = np.eye(3, dtype=np.float32)
    tri = np.array([[0, 1, 2]], dtype=np.int32)
    W = H = 21
    v = mkview(W=W, H=H, light=(0, 0, -1))
    o = oracle.render(v, pos, np.zeros_like(pos), col, tri)
    tri2 = [(p[0] / z, p[1] / z) for p in pos.astype(np.float64)]
    jj, ii = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    px = (2 * (ii.ravel() + 0.5) / W - 1) * 0.5
    py = (2 * (jj.ravel() + 0.5) / H - 1) * 0.5
    (ax, ay), (bx, by), (cx, cy) = tri2
    e0 = (cx - bx) * (py - by) - (cy - by) * (px - bx)
    e1 = (ax - cx) * (py - cy) - (ay - cy) * (px - cx)
    e2 = (bx - ax) * (py - ay) - (by - ay) * (px - ax)
    lam = np.stack([e0, e1, e2], 1) / (e0 + e1 + e2)[:, None]
    hit = o["id"] != BG
    assert hit.sum() > 50
    assert np.allclose(o["rgb"][hit], lam[hit], atol=1e-12)


@pytest.mark.parametrize("light", [(0.0, 0.0, -1.0), (0.6, -0.48, -0.64)])
def test_specular_flat_closed_form(oracle, light):
    """Blinn-Phong on a fronto-parallel triangle (normal (0, 0, -1) towards the
    camera): at every covered pixel rgb = c (k_a + k_d max(0, n.l)) +
    k_s max(0, n.h)^m with h = normalize(l - dir/|dir|), dir the pixel's ray."""
    pos, col, tri = _flat()
    k_s, m = 0.35, 24.0
    W = H = 11
    v = mkview(W=W, H=H, light=light, k_s=k_s, shininess=m)
    o = oracle.render(v, pos, np.zeros_like(pos), col, tri)
    l = np.array(light, dtype=np.float64) / np.linalg.norm(light)
    n = np.array([0.0, 0.0, -1.0])
    hit = np.nonzero(o["id"] == 0)[0]
    assert hit.size > 20
    for k in hit:
        i, j = k % W, k // W
        dvec = np.array([(2 * (i + 0.5) / W - 1) * 0.5, (2 * (j + 0.5) / H - 1) * 0.5, 1.0])
        hv = l - dvec / np.linalg.norm(dvec)
        hv /= np.linalg.norm(hv)
        want = np.array([0.2, 0.5, 0.8]) * (_f32(0.1) + _f32(0.9) * max(0.0, n @ l)) + _f32(k_s) * max(0.0, n @ hv) ** m
        assert np.allclose(o["rgb"][k], want, atol=1e-12)


def test_rolling_light(oracle):
    """The light follows the camera pose at the pixel time: with a 90 degree
    yaw over the frame, l(t) = normalize((1-t) R0 l + t R1 l)."""
    v = mkview(pose1=S.make_pose(S.rot_yaw(90.0)), light=(0.0, 0.0, -1.0))
    assert np.allclose(oracle.light(v, 0.0), [0, 0, -1], atol=1e-15)
    # R_yaw(90) = [[0,0,1],[0,1,0],[-1,0,0]] maps (0,0,-1) to (-1,0,0)
    assert np.allclose(oracle.light(v, 1.0), [-1, 0, 0], atol=1e-7)
    assert np.allclose(oracle.light(v, 0.5), np.array([-0.5, 0, -0.5]) / math.sqrt(0.5), atol=1e-7)


# --------------------------------------------------------------------------
# gradient: FP64 analytic vs central finite differences
# --------------------------------------------------------------------------

@pytest.mark.parametrize("mode,k_s", [(S.MODE_ROLLING, 0.0), (S.MODE_BOTH, 0.0), (S.MODE_BOTH, 0.4)])
def test_gradient_matches_finite_differences(oracle, mode, k_s):
    rng = np.random.default_rng(11 + mode)
    sc = S.random_triangles(40, 3, vel_sigma=0.05, offset=0.6)
    pose1 = S.make_pose(S.rot_pitch(1.0) @ S.rot_yaw(4.0), (0.02, 0.0, 0.0))
    v = mkview(W=40, H=32, mode=mode, pose1=pose1, fovea=(0.45, 0.55),
               light=tuple(np.array([-1.0, -1.0, -1.0]) / math.sqrt(3.0)), k_s=k_s, shininess=6.0)
    pos, vel, col = (a.astype(np.float64) for a in (sc.pos, sc.vel, sc.col))
    o = oracle.render(v, pos, vel, col, sc.tri, near=True)
    interior = (o["id"] != BG) & (o["bmin"] > 1e-3) & (o["gap"] > 1e-3) & (o["near"] > 1e-3)
    pix = np.nonzero(interior)[0]
    assert pix.size > 100
    g = rng.normal(size=(pix.size, 3))
    dc, dp, dv = oracle.grad(v, pos, vel, col, sc.tri, o["id"][pix], g, pix=pix)

    def loss(p_, v_, c_):
        r = oracle.render(v, p_, v_, c_, sc.tri, pix=pix)
        assert np.array_equal(r["id"], o["id"][pix])          # visibility held fixed
        return float((g * r["rgb"]).sum())

    h = 1e-4
    for name, arr, ana in (("col", col, dc), ("pos", pos, dp), ("vel", vel, dv)):
        fd = np.zeros_like(arr)
        idx = rng.choice(arr.size, size=24, replace=False)
        for k in idx:
            a1, a2 = arr.copy().ravel(), arr.copy().ravel()
            a1[k] += h
            a2[k] -= h
            args1 = {"col": (pos, vel, a1.reshape(arr.shape)), "pos": (a1.reshape(arr.shape), vel, col),
                     "vel": (pos, a1.reshape(arr.shape), col)}[name]
            args2 = {"col": (pos, vel, a2.reshape(arr.shape)), "pos": (a2.reshape(arr.shape), vel, col),
                     "vel": (pos, a2.reshape(arr.shape), col)}[name]
            fd.ravel()[k] = (loss(*args1) - loss(*args2)) / (2 * h)
        a = ana.ravel()[idx]
        f = fd.ravel()[idx]
        assert np.linalg.norm(a - f) <= 1e-6 * max(np.linalg.norm(f), 1e-12), name


# --------------------------------------------------------------------------
# regression fixture written by tests/golden/make_golden.py (oracle only)
# --------------------------------------------------------------------------

def test_golden_tiny_joint(oracle):
    import os
    from tests.golden.make_golden import golden_case
    path = os.path.join(os.path.dirname(__file__), "golden", "tiny_joint.txt")
    rows = np.loadtxt(path, comments="#")
    view, sc = golden_case()
    o = oracle.render(view, sc.pos, sc.vel, sc.col, sc.tri)
    assert np.array_equal(o["id"].astype(np.int64), rows[:, 1].astype(np.int64))
    hit = o["id"] != BG
    assert np.allclose(o["s"][hit], rows[hit, 2], rtol=1e-12)
