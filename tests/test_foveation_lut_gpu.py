"""A foveation function given by samples (Sec. 3.1.1, any monotonic p; Sec. 6,
lens distortion p = p_c o p_l) on the GPU against the FP64 oracle with the
same samples: frame parity, conservative bounds, the FP64 re-test, and the
display step (rendered with p_c o p_l, sampled back with p_c alone)."""
import dataclasses

import numpy as np
import pytest

from paper_1806_05385_gb300 import foveation as F
from paper_1806_05385_gb300 import scenes as S
from tests.parity_util import BG, compare
from tests.test_parity_gpu import gpu_frame, small_case
from tests.test_unfoveate_gpu import _check as check_display

pytestmark = pytest.mark.gpu

LENS = F.lens_samples(2.0, 0.22, 0.24, 1024)


def _lut_case(mode, seed=0, W=192, H=160, T=900, samples=LENS):
    sc, view = small_case(mode, seed=seed, W=W, H=H, T=T)
    return sc, dataclasses.replace(view, p_lut=samples)


@pytest.mark.parametrize("mode", [S.MODE_FOVEATED, S.MODE_BOTH])
@pytest.mark.parametrize("samples", [LENS, F.power_samples(3.0, 256)])
def test_sampled_p_frame_parity(pr, oracle, mode, samples):
    sc, view = _lut_case(mode, samples=samples)
    g = gpu_frame(pr, sc, view)
    o = oracle.render(view, sc.pos, sc.vel, sc.col, sc.tri)
    rep = compare(oracle, view, sc, o, g["id"], g["depth"], g["rgb"])
    assert rep["hit_frac"] > 0.05


@pytest.mark.parametrize("mode", [S.MODE_FOVEATED, S.MODE_BOTH])
def test_sampled_p_bounds_conservative(pr, oracle, mode):
    sc, view = _lut_case(mode, seed=3, W=176, H=144, T=700)
    g = gpu_frame(pr, sc, view, keep=True)
    box, tr = pr.pr_debug_bounds(g["scene"], sc.T)
    pr.pr_scene_free(g["scene"])
    o = oracle.render(view, sc.pos, sc.vel, sc.col, sc.tri)
    hit = np.nonzero(o["id"] != BG)[0]
    ids = o["id"][hit]
    i, j = hit % view.W, hit // view.W
    b = box[ids]
    assert ((i >= b[:, 0]) & (i <= b[:, 2]) & (j >= b[:, 1]) & (j <= b[:, 3])).all()


def test_sampled_p_fp64_retest_strict(pr, oracle):
    sc, view = _lut_case(S.MODE_BOTH, seed=11)
    g = gpu_frame(pr, sc, view, fp64=1)
    o = oracle.render(view, sc.pos, sc.vel, sc.col, sc.tri)
    compare(oracle, view, sc, o, g["id"], g["depth"], g["rgb"], fp64=True)


@pytest.mark.parametrize("method", ["mip", "projected"])
def test_lens_render_then_cortical_display(pr, oracle, method):
    """Sec. 6: render with p = p_c o p_l; sample back with p_c only, since the
    lens applies p_l optically."""
    sc, view = _lut_case(S.MODE_BOTH, seed=6, W=160, H=128, T=800)
    g = gpu_frame(pr, sc, view)
    img = g["rgb"].reshape(3, view.H, view.W)
    cortical = dataclasses.replace(view, p_lut=None, alpha=2.0)
    out = check_display(oracle, pr, cortical, img, 200, 160, method)
    assert np.isfinite(out).all()
    # the display step with the sampled map itself also matches the oracle
    check_display(oracle, pr, view, img, 200, 160, method)


def test_invalid_samples_are_rejected(pr):
    with pytest.raises(pr.PrError):
        pr.pr_foveation_create(np.array([0.0, 0.5, 0.5], np.float32))   # not strictly increasing
    with pytest.raises(pr.PrError):
        pr.pr_foveation_create(np.array([0.1, 0.5, 0.9], np.float32))   # p(0) != 0
    h = pr.pr_foveation_create(np.array([0.0, 0.7, 1.4], np.float32))
    pr.pr_foveation_free(h)
