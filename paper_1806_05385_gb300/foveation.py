"""Foveation functions given as samples (Sec. 3.1.1: p may be any monotonic
function, "inverted numerically in a pre-processing pass"; Sec. 6, "Lens
Distortion": p = p_c o p_l).

The library takes p as its values at d_k = k D / n, k = 0..n (D = sqrt(2)),
and interpolates linearly between them; its inverse is exact for that
interpolation.  These helpers make such samples:

* ``power_samples(alpha, n)``: the cortical power map p_c(d) = D (d/D)^alpha;
* ``lens_samples(alpha, k1, k2, n)``: the composition p = p_c o p_l with the
  radial barrel lens polynomial p_l(d) = d (1 + k1 d^2 + k2 d^4) (the form
  of the lens models HMD SDKs ship), both radial about the fovea as in the
  paper's composition.  Rendering uses p; the display step then samples back
  with p_c alone (a view with the power map), since p_l happens optically.
"""
from __future__ import annotations

import math

import numpy as np

D = math.sqrt(2.0)


def power_samples(alpha: float = 2.0, n: int = 1024) -> np.ndarray:
    d = np.arange(n + 1, dtype=np.float64) * (D / n)
    return (D * (d / D) ** alpha).astype(np.float32)


def lens_samples(alpha: float = 2.0, k1: float = 0.22, k2: float = 0.24, n: int = 1024) -> np.ndarray:
    if k1 < 0 or k2 < 0:
        raise ValueError("the barrel polynomial is monotone for k1, k2 >= 0")
    d = np.arange(n + 1, dtype=np.float64) * (D / n)
    dl = d * (1.0 + k1 * d * d + k2 * d ** 4)
    return (D * (dl / D) ** alpha).astype(np.float32)
