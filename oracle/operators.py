"""FP64 oracle operators: parallel-beam and fan-beam geometries, Joseph K / K^T,
finite differences D / D^T.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
from __future__ import annotations

import ctypes
import dataclasses
import math

import numpy as np

from . import _clib


@dataclasses.dataclass
class Geometry:
    """Parallel-beam geometry (Sec. 2, eq. (radon-def): rays u cos + v sin = s).

    theta: angles (float64); by default theta_a = a*pi/n_angles.
    row_branch[a] is 1 when the ray is stepped over image rows (|cos| >= |sin|,
    ties included).  For the default angles the test is done exactly on the
    integer a (4a <= n or 4a >= 3n); for user angles it is done on the FP64
    cos/sin values.
    """
    N: int
    n_angles: int
    n_det: int
    spacing: float = 1.0
    offset: float = 0.0
    theta: np.ndarray | None = None

    def __post_init__(self):
        if self.theta is None:
            self.theta = np.arange(self.n_angles, dtype=np.float64) * (math.pi / self.n_angles)
            a = np.arange(self.n_angles)
            rb = (4 * a <= self.n_angles) | (4 * a >= 3 * self.n_angles)
        else:
            self.theta = np.asarray(self.theta, dtype=np.float64)
            rb = np.abs(np.cos(self.theta)) >= np.abs(np.sin(self.theta))
        self.cos = np.ascontiguousarray(np.cos(self.theta))
        self.sin = np.ascontiguousarray(np.sin(self.theta))
        self.row_branch = np.ascontiguousarray(rb.astype(np.int32))

    @property
    def m(self) -> int:
        return self.n_angles * self.n_det

    @property
    def n(self) -> int:
        return self.N * self.N


@dataclasses.dataclass
class FanGeometry:
    """Fan-beam geometry with an equiangular (arc) detector (Sec. 4, "fan beam and cone
    beam geometry": the divergent-beam transform).

    Pixel coordinates as in Geometry (pixel (j, i) at u = i - (N-1)/2, v = (N-1)/2 - j).
    View a puts the source at S_a = R (-sin beta_a, cos beta_a), R = src_dist, with
    beta_a = 2.0 * pi * a / n_angles (that order of operations) unless beta is given.
    Channel t receives the ray leaving S_a at the fan angle gamma_t = (t - (n_det-1)/2) *
    pitch + offset, counted counter-clockwise from the central ray (S_a towards the
    centre).  That ray is the line u cos(theta) + v sin(theta) = s with theta = beta_a +
    gamma_t and s = R sin(gamma_t); it is stepped over rows when |cos theta| >= |sin theta|
    (tested on the FP64 values), with Joseph's interpolation and path-length weight as for
    the parallel beam.  cos, sin and s are computed per ray with the C library's cos / sin.
    """
    N: int
    n_angles: int
    n_det: int
    src_dist: float
    pitch: float
    offset: float = 0.0
    beta: np.ndarray | None = None

    def __post_init__(self):
        na, nd = self.n_angles, self.n_det
        if self.beta is None:
            self.beta = np.array([2.0 * math.pi * a / na for a in range(na)], dtype=np.float64)
        else:
            self.beta = np.asarray(self.beta, dtype=np.float64)
        cd = 0.5 * (nd - 1)
        self.gamma = np.array([(t - cd) * self.pitch + self.offset for t in range(nd)], dtype=np.float64)
        c = np.empty(na * nd)
        sn = np.empty(na * nd)
        s = np.empty(na * nd)
        rb = np.empty(na * nd, dtype=np.int32)
        R = float(self.src_dist)
        for a in range(na):
            for t in range(nd):
                th = float(self.beta[a]) + float(self.gamma[t])
                k = a * nd + t
                c[k] = math.cos(th)
                sn[k] = math.sin(th)
                s[k] = R * math.sin(float(self.gamma[t]))
                rb[k] = 1 if abs(c[k]) >= abs(sn[k]) else 0
        self.cos_r, self.sin_r, self.s_r, self.row_branch = c, sn, s, rb

    def source(self, a: int):
        """Source position of view a, (u, v)."""
        b = float(self.beta[a])
        return (-self.src_dist * math.sin(b), self.src_dist * math.cos(b))

    @property
    def m(self) -> int:
        return self.n_angles * self.n_det

    @property
    def n(self) -> int:
        return self.N * self.N


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _K_rays(x, g):
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(g.N, g.N)
    y = np.empty((g.n_angles, g.n_det), dtype=np.float64)
    _clib.lib().oracle_joseph_forward_rays(g.N, g.m, _dp(g.cos_r), _dp(g.sin_r), _dp(g.s_r),
                                           g.row_branch.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                           _dp(x), _dp(y))
    return y


def _KT_rays(y, g):
    y = np.ascontiguousarray(y, dtype=np.float64).reshape(g.n_angles, g.n_det)
    x = np.empty((g.N, g.N), dtype=np.float64)
    _clib.lib().oracle_joseph_transpose_rays(g.N, g.m, _dp(g.cos_r), _dp(g.sin_r), _dp(g.s_r),
                                             g.row_branch.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                             _dp(y), _dp(x))
    return x


def fan_projector(N: int, n_angles: int, n_det: int, src_dist: float, pitch: float, offset: float = 0.0):
    """x -> K x for the fan beam with default views (for the seeded input generator)."""
    g = FanGeometry(N, n_angles, n_det, src_dist, pitch, offset)
    return lambda x: K(x, g)


def K(x: np.ndarray, g: Geometry) -> np.ndarray:
    """Joseph forward projection y = K x, y[a, t] (float64)."""
    if isinstance(g, FanGeometry):
        return _K_rays(x, g)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(g.N, g.N)
    y = np.empty((g.n_angles, g.n_det), dtype=np.float64)
    _clib.lib().oracle_joseph_forward(g.N, g.n_angles, g.n_det, _dp(g.cos), _dp(g.sin),
                                      g.row_branch.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                      g.spacing, g.offset, _dp(x), _dp(y))
    return y


def projector(N: int, n_angles: int, n_det: int, spacing: float = 1.0, offset: float = 0.0):
    """x -> K x for the default angles: the projector passed to the seeded input
    generator, which makes b = K x_true + noise."""
    g = Geometry(N, n_angles, n_det, spacing=spacing, offset=offset)
    return lambda x: K(x, g)


def KT(y: np.ndarray, g: Geometry) -> np.ndarray:
    """Exact transpose x = K^T y of the Joseph projector (float64, N x N)."""
    if isinstance(g, FanGeometry):
        return _KT_rays(y, g)
    y = np.ascontiguousarray(y, dtype=np.float64).reshape(g.n_angles, g.n_det)
    x = np.empty((g.N, g.N), dtype=np.float64)
    _clib.lib().oracle_joseph_transpose(g.N, g.n_angles, g.n_det, _dp(g.cos), _dp(g.sin),
                                        g.row_branch.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                        g.spacing, g.offset, _dp(y), _dp(x))
    return x


# ---------------------------------------------------------------------------
# Finite differences (Sec. 2): D_n has rows [1, -1], so (D_n x)_i = x_i - x_{i+1},
# D_n in R^{(n-1) x n}.  In 2D, D_2 = [I (x) D_n ; D_n (x) I] acting on the
# row-major image: horizontal differences (along a row) and vertical ones.
# ---------------------------------------------------------------------------

def D(x: np.ndarray):
    """Return (dh, dv): dh[j, i] = x[j,i]-x[j,i+1] (N x N-1), dv[j, i] = x[j,i]-x[j+1,i] (N-1 x N)."""
    x = np.asarray(x, dtype=np.float64)
    return x[:, :-1] - x[:, 1:], x[:-1, :] - x[1:, :]


def DT(dh: np.ndarray, dv: np.ndarray) -> np.ndarray:
    """Transpose of D: D^T (dh, dv), N x N."""
    N = dh.shape[0]
    out = np.zeros((N, N), dtype=np.float64)
    out[:, :-1] += dh
    out[:, 1:] -= dh
    out[:-1, :] += dv
    out[1:, :] -= dv
    return out


def D1_matrix(n: int) -> np.ndarray:
    """Dense D_n (Sec. 2): (n-1) x n with 1 on the diagonal and -1 above it."""
    Dn = np.zeros((n - 1, n))
    for i in range(n - 1):
        Dn[i, i] = 1.0
        Dn[i, i + 1] = -1.0
    return Dn


def dense_of(op, n_in: int) -> np.ndarray:
    """Dense matrix of a linear map given as a function on flat vectors."""
    cols = []
    for k in range(n_in):
        e = np.zeros(n_in)
        e[k] = 1.0
        cols.append(np.ravel(op(e)))
    return np.stack(cols, axis=1)
