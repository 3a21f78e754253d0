"""The seeded input generators (no GPU): meshes are closed and consistently
oriented, and every workload has the sizes, field of view, eye separation,
motion and value ranges of its recipe, reproducibly for a seed."""
import math

import numpy as np
import pytest

from paper_1806_05385_gb300 import scenes as S


def _closed_and_oriented(v, f):
    """Every directed edge appears once and its reverse once (a closed,
    consistently oriented surface); returns the signed volume."""
    edges = {}
    for a, b, c in f:
        for e in ((a, b), (b, c), (c, a)):
            edges[e] = edges.get(e, 0) + 1
    assert all(n == 1 for n in edges.values())
    assert all((b, a) in edges for a, b in edges)
    p = v[f]
    return float(np.einsum("ij,ij->i", p[:, 0], np.cross(p[:, 1], p[:, 2])).sum() / 6.0)


@pytest.mark.parametrize("k", [0, 1, 2, 3])
def test_icosphere(k):
    v, f = S.icosphere(k)
    assert f.shape == (20 * 4 ** k, 3)
    assert np.allclose(np.linalg.norm(v, axis=1), 1.0)
    assert len(v) - 3 * len(f) // 2 + len(f) == 2  # Euler: V - E + F = 2
    vol = _closed_and_oriented(v, f)
    # inscribed in the unit sphere, approaching its volume with subdivision
    assert 0.6 * 4 * math.pi / 3 < abs(vol) < 4 * math.pi / 3
    if k == 3:
        assert abs(vol) > 0.98 * 4 * math.pi / 3


def test_unit_box_and_ground_plane():
    v, f = S.unit_box()
    assert f.shape == (12, 3)
    assert abs(_closed_and_oriented(v, f)) == pytest.approx(8.0)
    gv, gf = S.ground_plane(5, 7, 1.6, (-20.0, 20.0), (0.5, 40.5))
    assert gf.shape == (2 * 5 * 7, 3) and gv.shape == (6 * 8, 3)
    assert np.all(gv[:, 1] == 1.6)
    assert gv[:, 0].min() == -20.0 and gv[:, 2].max() == 40.5
    # the two triangles of every quad cover it: total area = plane area
    p = gv[gf]
    area = 0.5 * np.linalg.norm(np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]), axis=1).sum()
    assert area == pytest.approx(40.0 * 40.0)


def _rotation_angle(R):
    return math.degrees(math.acos(max(-1.0, min(1.0, (np.trace(R) - 1.0) / 2.0))))


def test_config_small_recipe():
    sc, (view,) = S.config_small(seed=0)
    assert sc.T == 1000 and sc.pos.shape == (3000, 3)
    assert np.all(np.abs(sc.pos[:, :2]) <= 1.0) and np.all((sc.pos[:, 2] >= 2.0) & (sc.pos[:, 2] <= 10.0))
    assert abs(float(sc.vel.std()) - 0.05) < 0.005
    assert np.all((sc.col >= 0.0) & (sc.col <= 1.0))
    assert (view.W, view.H, view.mode, view.tan_x, view.tan_y) == (256, 256, S.MODE_ROLLING, 0.5, 0.5)
    assert np.array_equal(view.pose0, np.eye(4, dtype=np.float32))
    assert _rotation_angle(view.pose1[:3, :3].astype(np.float64)) == pytest.approx(2.0, abs=1e-3)


def test_config_hmd_recipe():
    sc, views = S.config_hmd(seed=2)
    assert sc.T == 200 * 1280 + 10000
    assert len(views) == 2
    for v in views:
        assert (v.W, v.H, v.mode, v.alpha) == (1440, 1600, S.MODE_BOTH, 2.0)
        assert v.tan_x == pytest.approx(math.tan(math.radians(50.0)))
        assert v.tan_y / v.tan_x == pytest.approx(1600 / 1440)  # square pixels
        assert all(0.2 <= c <= 0.8 for c in v.fovea)
        assert np.allclose(v.pose0[:3, :3], np.eye(3))
        # head yaw 3 and pitch 1 degrees over the frame
        R1 = v.pose1[:3, :3].astype(np.float64)
        assert np.allclose(R1, S.rot_pitch(1.0) @ S.rot_yaw(3.0), atol=1e-6)
    # IPD 0.064 along the camera x axis
    assert views[1].pose0[0, 3] - views[0].pose0[0, 3] == pytest.approx(-0.064)
    assert views[0].pose0[1, 3] == views[0].pose0[2, 3] == 0.0
    # 200 icospheres of 642 vertices each, then the ground plane
    nv = 200 * 642
    obj_pos, obj_vel = sc.pos[:nv].reshape(200, 642, 3), sc.vel[:nv].reshape(200, 642, 3)
    assert np.all(obj_vel == obj_vel[:, :1])  # one velocity per object
    speed = np.linalg.norm(obj_vel[:, 0], axis=1)
    assert speed.max() <= 0.3 + 1e-6 and speed.min() >= 0.0
    assert obj_pos[..., 2].min() >= 1.0 - 1e-5  # every object beyond depth 1
    assert obj_pos[..., 2].max() <= 30.0 + 1.5 + 1e-4
    radius = np.linalg.norm(obj_pos - obj_pos.mean(axis=1, keepdims=True), axis=2).max(axis=1)
    assert radius.min() >= 0.2 - 1e-3 and radius.max() <= 1.5 + 1e-3
    assert np.all(sc.vel[nv:] == 0.0) and np.allclose(sc.pos[nv:, 1], 1.6)
    # reproducible for a seed, different for another
    sc2, views2 = S.config_hmd(seed=2)
    assert np.array_equal(sc.pos, sc2.pos) and views[0].fovea == views2[0].fovea
    assert not np.array_equal(sc.pos, S.config_hmd(seed=3)[0].pos)


def test_config_large_recipe():
    sc, views = S.config_large(seed=3)
    assert sc.T == 1_000_000
    assert [(v.W, v.H) for v in views] == [(2160, 2160)] * 2
    assert int(sc.tri.max()) < sc.V
    moving = np.linalg.norm(sc.vel, axis=1) > 0
    assert 0.3 < moving.mean() < 0.7  # about half the instances move


def test_config_batched_recipe():
    pairs = S.config_batched(seed=4)
    assert len(pairs) == 64
    sides = [v.W for _, v in pairs]
    Ts = [sc.T for sc, _ in pairs]
    assert all(v.W == v.H for _, v in pairs)
    assert 512 <= min(sides) and max(sides) <= 2160
    assert 1000 <= min(Ts) and max(Ts) <= 500_000
    assert {v.mode for _, v in pairs} == {S.MODE_CLASSIC, S.MODE_ROLLING, S.MODE_FOVEATED, S.MODE_BOTH}
    # log-uniform sizes: the geometric mean sits near the middle of the range
    assert math.exp(np.mean(np.log(Ts))) == pytest.approx(math.sqrt(1000 * 500_000), rel=0.5)


def test_config_diff_recipe():
    sc, view, tgt = S.config_diff(seed=5)
    assert sc.T == 10_000 and (view.W, view.H, view.mode) == (512, 512, S.MODE_BOTH)
    # vertices within 0.15 of their triangle's centre (per axis): edges <= 0.3
    p = sc.pos[sc.tri]
    assert np.abs(p - p.mean(axis=1, keepdims=True)).max() <= 0.3 + 1e-6
    for a, b in ((sc.pos, tgt.pos), (sc.vel, tgt.vel)):
        assert abs(float((b - a).std()) - 0.01) < 0.001
    assert np.all((tgt.col >= 0.0) & (tgt.col <= 1.0)) and np.array_equal(sc.tri, tgt.tri)


def test_sample_pixels():
    idx = S.sample_pixels(1440, 1600, 1 << 16, 4, 64, seed=7)
    assert np.all(np.diff(idx) > 0) and idx.min() >= 0 and idx.max() < 1440 * 1600
    assert len(idx) >= 4 * 64 * 64  # the windows alone
    assert np.array_equal(idx, S.sample_pixels(1440, 1600, 1 << 16, 4, 64, seed=7))


def test_config_batched_span_recipe():
    """The batch that spans the 64-view workload's extremes: 1k and 500k
    triangles at its ends (geometric in between), sides 512..2160 (each used
    once), every mode twice and every tile size, reproducible per seed."""
    cases = S.config_batched_span(seed=4)
    assert len(cases) == 8
    Ts = [sc.T for sc, _, _ in cases]
    assert Ts[0] == 1000 and Ts[-1] == 500_000 and all(a < b for a, b in zip(Ts, Ts[1:]))
    sides = sorted(v.W for _, v, _ in cases)
    assert sides[0] == 512 and sides[-1] == 2160 and len(set(sides)) == 8
    assert all(v.W == v.H for _, v, _ in cases)
    assert sorted(v.mode for _, v, _ in cases) == [0, 0, 1, 1, 2, 2, 3, 3]
    assert {t for _, _, t in cases} == {8, 16, 32}
    again = S.config_batched_span(seed=4)
    for (a, va, ta), (b, vb, tb) in zip(cases, again):
        assert np.array_equal(a.pos, b.pos) and va.W == vb.W and ta == tb
