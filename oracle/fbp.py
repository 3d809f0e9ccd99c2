"""FP64 oracle for the Ram-Lak filtered backprojection used as a warm start
(not in the paper).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Ram-Lak kernel for bin pitch tau (Kak and Slaney, discrete ramp filter):
h(0) = 1/(4 tau^2), h(n) = 0 for even n != 0, h(n) = -1/(n^2 pi^2 tau^2) for odd n.
Each sinogram row is filtered by q = tau (h * b) (direct convolution), then
x = (pi / n_angles) K^T q with the oracle's exact transpose of the projector.
"""
from __future__ import annotations

import math

import numpy as np

from .operators import Geometry, KT


def ramlak(n_det: int, tau: float = 1.0) -> np.ndarray:
    """h(n) for n = -(n_det-1) .. (n_det-1)."""
    n = np.arange(-(n_det - 1), n_det)
    h = np.zeros(n.size)
    h[n == 0] = 1.0 / (4.0 * tau * tau)
    odd = (n % 2) != 0
    h[odd] = -1.0 / (n[odd].astype(np.float64) ** 2 * math.pi ** 2 * tau * tau)
    return h


def ramp_filter(b: np.ndarray, tau: float = 1.0) -> np.ndarray:
    b = np.asarray(b, dtype=np.float64)
    n_det = b.shape[1]
    h = ramlak(n_det, tau)
    out = np.empty_like(b)
    for a in range(b.shape[0]):
        out[a] = tau * np.convolve(b[a], h)[n_det - 1:2 * n_det - 1]
    return out


def fbp(b: np.ndarray, g: Geometry) -> np.ndarray:
    q = ramp_filter(np.asarray(b).reshape(g.n_angles, g.n_det), g.spacing)
    return (math.pi / g.n_angles) * KT(q, g)
