"""Seeded synthetic scenes and views shaped like head-mounted-display workloads.

This module only *constructs inputs*: vertex positions, per-frame vertex
velocities, per-vertex colours, triangle indices, the two camera poses that
bracket the frame interval, the fovea and the display parameters.  It holds
none of the rasterization arithmetic, so both the CUDA path and the FP64
oracle can be fed from it without sharing any of the method's code.

Conventions (shared by every consumer of these arrays):

* camera: x right, y down, z forward; a pose is a row-major 4x4 rigid
  world->camera transform ``[R | T]``; ``pose0`` holds at time 0 and
  ``pose1`` at time 1 of the frame interval (the start and end model-view
  matrices of Sec. 3.2, "Bounding").
* a vertex moves linearly over the frame: world position ``p + t * v``
  (Sec. 3.1.2, third display property).
* ``mode``: 0 classic, 1 rolling, 2 foveated, 3 both (Sec. 3.1.1-3.1.3).
* ``d``: rolling skew direction of ``r(x) = x . d`` (Sec. 3.1.2); ``alpha``:
  exponent of the power foveation ``p(d) = d^alpha`` (Sec. 5.1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MODE_CLASSIC, MODE_ROLLING, MODE_FOVEATED, MODE_BOTH = 0, 1, 2, 3
MODE_NAMES = {"classic": 0, "rolling": 1, "foveated": 2, "both": 3}


@dataclass
class Scene:
    pos: np.ndarray  # float32 [V,3] world positions at t=0
    vel: np.ndarray  # float32 [V,3] world displacement over the frame
    col: np.ndarray  # float32 [V,3] per-vertex RGB albedo in [0,1]
    tri: np.ndarray  # int32   [T,3] vertex indices

    @property
    def V(self) -> int:
        return int(self.pos.shape[0])

    @property
    def T(self) -> int:
        return int(self.tri.shape[0])


@dataclass
class View:
    W: int
    H: int
    tan_x: float
    tan_y: float
    pose0: np.ndarray  # float32 [4,4]
    pose1: np.ndarray  # float32 [4,4]
    mode: int = MODE_ROLLING
    fovea: tuple = (0.5, 0.5)
    alpha: float = 2.0
    d: tuple = (1.0, 0.0)
    z_near: float = 1e-3
    light_w: tuple = field(default_factory=lambda: tuple((np.array([-1.0, -1.0, -1.0]) / math.sqrt(3.0)).tolist()))
    k_a: float = 0.1
    k_d: float = 0.9
    k_s: float = 0.0        # rolling specular (Blinn-Phong) weight; 0: none
    shininess: float = 1.0
    p_lut: object = None    # optional samples of an arbitrary monotone p (float32 [n + 1]) instead of the power map


# ----------------------------------------------------------------------------
# poses
# ----------------------------------------------------------------------------

def rot_yaw(deg: float) -> np.ndarray:
    """Rotation about the camera's vertical (y) axis by ``deg`` degrees."""
    a = math.radians(deg)
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]], dtype=np.float64)


def rot_pitch(deg: float) -> np.ndarray:
    """Rotation about the camera's horizontal (x) axis by ``deg`` degrees."""
    a = math.radians(deg)
    c, s = math.cos(a), math.sin(a)
    return np.array([[1.0, 0.0, 0.0], [0.0, c, -s], [0.0, s, c]], dtype=np.float64)


def make_pose(R: np.ndarray, T=(0.0, 0.0, 0.0)) -> np.ndarray:
    M = np.eye(4, dtype=np.float64)
    M[:3, :3] = R
    M[:3, 3] = T
    return M.astype(np.float32)


def head_poses(yaw_deg: float, pitch_deg: float, eye_x: float = 0.0):
    """World->camera poses of one eye whose head rotates from identity to
    ``pitch @ yaw`` over the frame; the eye sits at ``eye_x`` along the head's
    x axis (so a point at the eye maps to the camera origin)."""
    R1 = rot_pitch(pitch_deg) @ rot_yaw(yaw_deg)
    T = (-eye_x, 0.0, 0.0)
    return make_pose(np.eye(3), T), make_pose(R1, T)


# ----------------------------------------------------------------------------
# meshes
# ----------------------------------------------------------------------------

def icosphere(subdiv: int):
    """Unit icosphere: 20 * 4**subdiv faces, shared vertices."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    verts = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
             (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
             (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    verts = [np.array(v, dtype=np.float64) / np.linalg.norm(v) for v in verts]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(subdiv):
        cache = {}

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    return np.array(verts, dtype=np.float64), np.array(faces, dtype=np.int32)


def unit_box():
    """Axis-aligned cube [-1,1]^3: 8 vertices, 12 triangles."""
    v = np.array([[x, y, z] for x in (-1, 1) for y in (-1, 1) for z in (-1, 1)], dtype=np.float64)
    f = np.array([[0, 1, 3], [0, 3, 2], [4, 6, 7], [4, 7, 5],
                  [0, 4, 5], [0, 5, 1], [2, 3, 7], [2, 7, 6],
                  [0, 2, 6], [0, 6, 4], [1, 5, 7], [1, 7, 3]], dtype=np.int32)
    return v, f


def ground_plane(nx: int, nz: int, y: float, x_range, z_range):
    """Grid of nx*nz quads (2 triangles each) in the plane at height ``y``."""
    xs = np.linspace(x_range[0], x_range[1], nx + 1)
    zs = np.linspace(z_range[0], z_range[1], nz + 1)
    X, Z = np.meshgrid(xs, zs, indexing="xy")
    v = np.stack([X.ravel(), np.full(X.size, y), Z.ravel()], 1)
    f = []
    for iz in range(nz):
        for ix in range(nx):
            a = iz * (nx + 1) + ix
            b, c, d = a + 1, a + nx + 1, a + nx + 2
            f += [(a, b, d), (a, d, c)]
    return v, np.array(f, dtype=np.int32)


def _concat(parts):
    pos, vel, col, tri = [], [], [], []
    base = 0
    for p, v, c, t in parts:
        pos.append(p)
        vel.append(v)
        col.append(c)
        tri.append(t + base)
        base += p.shape[0]
    return Scene(np.concatenate(pos).astype(np.float32), np.concatenate(vel).astype(np.float32),
                 np.concatenate(col).astype(np.float32), np.concatenate(tri).astype(np.int32))


def _random_direction(rng):
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

def random_triangles(T: int, seed: int, vel_sigma: float = 0.05, offset: float | None = None) -> Scene:
    """``T`` triangles with three independent vertices each.

    ``offset is None``: every vertex uniform in [-1,1]^2 x [2,10].
    ``offset = a``: a centre uniform in that box and each vertex at the centre
    plus U[-a,a]^3 (small triangles).  Per-vertex velocity N(0, vel_sigma),
    per-vertex colour U[0,1]."""
    rng = np.random.default_rng(seed)
    lo = np.array([-1.0, -1.0, 2.0])
    hi = np.array([1.0, 1.0, 10.0])
    if offset is None:
        pos = rng.uniform(lo, hi, size=(3 * T, 3))
    else:
        cen = rng.uniform(lo, hi, size=(T, 3))
        pos = np.repeat(cen, 3, axis=0) + rng.uniform(-offset, offset, size=(3 * T, 3))
    vel = rng.normal(0.0, vel_sigma, size=(3 * T, 3))
    col = rng.uniform(0.0, 1.0, size=(3 * T, 3))
    tri = np.arange(3 * T, dtype=np.int32).reshape(T, 3)
    return Scene(pos.astype(np.float32), vel.astype(np.float32), col.astype(np.float32), tri)


def instance_scene(rng, T_target: int, tan_x: float, tan_y: float, kinds=("ico3",),
                   radius=(0.2, 1.5), log_size=False, z_range=(1.0, 30.0), move_frac=1.0,
                   vmax=0.3, ground: int = 0) -> Scene:
    """Objects (icospheres/boxes) placed uniformly in the view frustum with
    centre depth U[z_range[0] + bounding radius, z_range[1]] (so every
    object lies entirely beyond z_range[0]), each with one linear velocity
    (uniform direction, |v| ~ U[0, vmax]); instances are added until
    ``T_target`` triangles are reached (the last one truncated).  ``ground`` > 0 adds a ground plane of
    that many triangles at y = +1.6 (y points down)."""
    meshes = {"ico3": icosphere(3), "ico2": icosphere(2), "box": unit_box()}
    parts = []
    total = 0
    while total < T_target:
        kind = kinds[int(rng.integers(len(kinds)))]
        v0, f0 = meshes[kind]
        if log_size:
            r = math.exp(rng.uniform(math.log(radius[0]), math.log(radius[1])))
        else:
            r = rng.uniform(*radius)
        # the nearest point of the object stays at depth >= z_range[0]: no
        # object encloses the eye or reaches through the near plane
        rb = r * float(np.linalg.norm(v0, axis=1).max())
        z = rng.uniform(z_range[0] + rb, max(z_range[1], z_range[0] + rb))
        cx = rng.uniform(-z * tan_x, z * tan_x)
        cy = rng.uniform(-z * tan_y, z * tan_y)
        p = v0 * r + np.array([cx, cy, z])
        if rng.uniform() < move_frac:
            vel = _random_direction(rng) * rng.uniform(0.0, vmax)
        else:
            vel = np.zeros(3)
        f = f0
        if total + f.shape[0] > T_target:
            f = f[: T_target - total]
        c = rng.uniform(0.0, 1.0, size=(p.shape[0], 3))
        parts.append((p, np.repeat(vel[None], p.shape[0], 0), c, f))
        total += f.shape[0]
    if ground:
        nq = ground // 2
        nx = int(round(math.sqrt(nq / 2)))
        nz = nq // nx
        gv, gf = ground_plane(nx, nz, 1.6, (-20.0, 20.0), (0.5, 40.5))
        parts.append((gv, np.zeros_like(gv), rng.uniform(0.0, 1.0, size=gv.shape), gf))
    return _concat(parts)


def config_small(seed: int = 0):
    """256x256 rolling frame of 1,000 random triangles (vertices U([-1,1]^2 x
    [2,10]), velocity N(0,0.05) per frame), camera yaw 0->2 degrees,
    t(x) = x/W, identity foveation."""
    sc = random_triangles(1000, seed)
    p0, p1 = head_poses(2.0, 0.0)
    view = View(W=256, H=256, tan_x=0.5, tan_y=0.5, pose0=p0, pose1=p1, mode=MODE_ROLLING)
    return sc, [view]


def hmd_fov(W: int, H: int, hfov_deg: float = 100.0):
    tan_x = math.tan(math.radians(hfov_deg / 2.0))
    return tan_x, tan_x * H / W


def config_hmd(seed: int = 2, W: int = 1440, H: int = 1600, n_objects: int = 200):
    """Stereo foveated+rolling frame: 1440x1600 per eye, 100 degree horizontal
    FOV, 200 icospheres (subdivision 3, radius r ~ U[0.2,1.5], centre depth
    U[1 + r, 30]) plus
    a 10,000-triangle ground plane, per-object velocity |v| <= 0.3 per frame,
    head yaw 0->3 and pitch 0->1 degrees, IPD 0.064, fovea U[0.2,0.8]^2 per
    eye, power foveation alpha = 2."""
    rng = np.random.default_rng(seed)
    tx, ty = hmd_fov(W, H)
    sc = instance_scene(rng, n_objects * 1280, tx, ty, kinds=("ico3",), ground=10000)
    views = []
    for eye in (-0.032, 0.032):
        p0, p1 = head_poses(3.0, 1.0, eye)
        fov = tuple(rng.uniform(0.2, 0.8, size=2).tolist())
        views.append(View(W=W, H=H, tan_x=tx, tan_y=ty, pose0=p0, pose1=p1, mode=MODE_BOTH,
                          fovea=fov, alpha=2.0))
    return sc, views


def config_large(seed: int = 3, side: int = 2160, T: int = 1_000_000):
    """Large stereo frame: 2160x2160 per eye, 1M triangles of icosphere
    (subdivision 2) and box instances (50/50), log-uniform size 1e-3..1, half
    of the instances moving (|v| <= 0.3), foveated+rolling."""
    rng = np.random.default_rng(seed)
    tx, ty = hmd_fov(side, side)
    sc = instance_scene(rng, T, tx, ty, kinds=("ico2", "box"), radius=(1e-3, 1.0), log_size=True,
                        move_frac=0.5)
    views = []
    for eye in (-0.032, 0.032):
        p0, p1 = head_poses(3.0, 1.0, eye)
        fov = tuple(rng.uniform(0.2, 0.8, size=2).tolist())
        views.append(View(W=side, H=side, tan_x=tx, tan_y=ty, pose0=p0, pose1=p1, mode=MODE_BOTH,
                          fovea=fov, alpha=2.0))
    return sc, views


def config_batched(seed: int = 4, n_views: int = 64, T_range=(1_000, 500_000), side_range=(512, 2160),
                   scale: float = 1.0):
    """``n_views`` independent views, each with its own scene: triangle count
    log-uniform in ``T_range``, square resolution with log-uniform side in
    ``side_range``, mode uniform over {classic, rolling, foveated, both},
    fovea U[0.2,0.8]^2.  ``scale`` < 1 shrinks triangle counts and sides for
    small test cases."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_views):
        T = int(math.exp(rng.uniform(math.log(T_range[0]), math.log(T_range[1]))) * scale)
        side = int(math.exp(rng.uniform(math.log(side_range[0]), math.log(side_range[1]))) * math.sqrt(scale))
        side = max(side, 16)
        T = max(T, 16)
        mode = int(rng.integers(4))
        tx, ty = hmd_fov(side, side, 90.0)
        sc = instance_scene(rng, T, tx, ty, kinds=("ico2", "box"), radius=(0.01, 1.0), log_size=True,
                            move_frac=0.5)
        yaw = rng.uniform(0.0, 3.0)
        pitch = rng.uniform(0.0, 1.0)
        p0, p1 = head_poses(yaw, pitch)
        fov = tuple(rng.uniform(0.2, 0.8, size=2).tolist())
        out.append((sc, View(W=side, H=side, tan_x=tx, tan_y=ty, pose0=p0, pose1=p1, mode=mode,
                             fovea=fov, alpha=2.0)))
    return out


def config_batched_span(seed: int = 4, n_views: int = 8, T_range=(1_000, 500_000), side_range=(512, 2160),
                        tiles=(8, 16, 32)):
    """A batch shaped like the 64-view workload that spans its extremes:
    view k has T_k = T_lo (T_hi/T_lo)^(k/(n-1)) triangles (so the first has
    1k and the last 500k), a square side taken from the same geometric
    sequence over ``side_range`` in a seeded order, mode k mod 4 (every mode
    twice for 8 views) and tile size tiles[k mod 3]; scenes, fovea and head
    motion follow the 64-view recipe.  Returns (scene, view, tile) triples."""
    rng = np.random.default_rng(seed)
    n = n_views
    Ts = [int(round(T_range[0] * (T_range[1] / T_range[0]) ** (k / (n - 1)))) for k in range(n)]
    sides = [int(round(side_range[0] * (side_range[1] / side_range[0]) ** (k / (n - 1)))) for k in range(n)]
    sides = [sides[k] for k in rng.permutation(n)]
    out = []
    for k in range(n):
        tx, ty = hmd_fov(sides[k], sides[k], 90.0)
        sc = instance_scene(rng, Ts[k], tx, ty, kinds=("ico2", "box"), radius=(0.01, 1.0), log_size=True,
                            move_frac=0.5)
        p0, p1 = head_poses(rng.uniform(0.0, 3.0), rng.uniform(0.0, 1.0))
        fov = tuple(rng.uniform(0.2, 0.8, size=2).tolist())
        out.append((sc, View(W=sides[k], H=sides[k], tan_x=tx, tan_y=ty, pose0=p0, pose1=p1, mode=k % 4,
                             fovea=fov, alpha=2.0), tiles[k % len(tiles)]))
    return out


def config_diff(seed: int = 5, W: int = 512, H: int = 512, T: int = 10_000, sigma: float = 0.01):
    """Differentiable case: 512x512 rolling+foveated, 10k small triangles
    (centres as the small config, vertex offsets U[-0.15,0.15]^3).  Returns
    the scene, the view and a target scene whose colours, positions and
    velocities are perturbed by N(0, sigma)."""
    rng = np.random.default_rng(seed)
    sc = random_triangles(T, seed, offset=0.15)
    p0, p1 = head_poses(2.0, 0.0)
    fov = tuple(rng.uniform(0.3, 0.7, size=2).tolist())
    view = View(W=W, H=H, tan_x=0.5, tan_y=0.5, pose0=p0, pose1=p1, mode=MODE_BOTH, fovea=fov, alpha=2.0)
    tgt = Scene((sc.pos + rng.normal(0, sigma, sc.pos.shape)).astype(np.float32),
                (sc.vel + rng.normal(0, sigma, sc.vel.shape)).astype(np.float32),
                np.clip(sc.col + rng.normal(0, sigma, sc.col.shape), 0.0, 1.0).astype(np.float32),
                sc.tri.copy())
    return sc, view, tgt


def sample_pixels(W: int, H: int, n_uniform: int, n_windows: int, win: int, seed: int) -> np.ndarray:
    """Seeded pixel subset (linear indices j*W+i, sorted, unique): ``n_uniform``
    uniform pixels plus ``n_windows`` square windows of side ``win``."""
    rng = np.random.default_rng(seed)
    idx = [rng.integers(0, W * H, size=n_uniform)]
    for _ in range(n_windows):
        i0 = int(rng.integers(0, max(1, W - win)))
        j0 = int(rng.integers(0, max(1, H - win)))
        jj, ii = np.meshgrid(np.arange(j0, min(H, j0 + win)), np.arange(i0, min(W, i0 + win)), indexing="ij")
        idx.append((jj * W + ii).ravel())
    return np.unique(np.concatenate(idx)).astype(np.int64)
