"""FP64 oracle for 3-D cone-beam NCS on a circular orbit (Sec. 4, "fan beam and cone beam
geometry": the 3-D divergent-beam transform, with the analogous 3-D circulant approximations
of eq. (H-fan) for K^T K and of eq. (circ_D) for D^T D).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Volume x[k, j, i]: Nz slices of N x N, voxel centre (u, v, w) = (i - (N-1)/2, (N-1)/2 - j,
k - (Nz-1)/2) in voxel units.  Sinogram y[a, r, t]: view a, detector row r, channel t.

Readings (the paper gives no cone-beam formulas; its cone-beam data set is absent):
  * the source circles in the plane w = 0 as in the fan beam (FanGeometry: S_a, fan angle
    gamma_t of channel t); the detector is cylindrical: row r sees the rays whose slope
    sigma_r = (r - (n_rows-1)/2) * row_pitch + row_offset is the rise in w per unit of in-plane
    distance from the source, so the in-plane trace of every ray of channel t is the fan ray
    of channel t;
  * Joseph's method in 3-D: the ray is stepped over the in-plane lines of its in-plane trace
    (rows or columns, the fan-beam rule), interpolated bilinearly in the other in-plane index
    and the slice index, and weighted by the path length per step sqrt(1 + sigma^2)/|cos|
    (or /|sin|); this needs |sigma| < 1/sqrt(2) so that the slice index never changes by more
    than one per step (the in-plane step is at most sqrt(2) long);
  * D = (D_x, D_y, D_z), the forward differences of Sec. 2 along each axis; TV is anisotropic
    (sum of |.|) or isotropic (per-voxel l2 norm of the three differences, zero at the last
    index of each axis);
  * M = gamma I + alpha C with C's eigenvalues alpha H_R + (beta^2/alpha) H_D (eq. (H-fan) in
    least-squares form for H_R over probe volumes, DC entry ||K 1||^2/||1||^2; H_D =
    4 (sin^2(pi p/N) + sin^2(pi q/N) + sin^2(pi l/Nz))), on an N x N x Nz periodic grid.
The iteration is eq. (NCS) with the updates of Sec. 4.1 written for these blocks.
"""
from __future__ import annotations

import ctypes
import dataclasses

import numpy as np

from . import _clib
from . import prox
from .operators import FanGeometry
from .solvers import splitmix64_uniform


@dataclasses.dataclass
class ConeGeometry:
    """Circular-orbit cone beam with a cylindrical detector (see the module notes)."""
    N: int
    Nz: int
    n_views: int
    n_rows: int
    n_det: int
    src_dist: float
    pitch: float
    row_pitch: float
    offset: float = 0.0
    row_offset: float = 0.0
    beta: np.ndarray | None = None

    def __post_init__(self):
        self.fan = FanGeometry(self.N, self.n_views, self.n_det, self.src_dist, self.pitch, self.offset,
                               beta=self.beta)
        self.sigma = np.array([(r - 0.5 * (self.n_rows - 1)) * self.row_pitch + self.row_offset
                               for r in range(self.n_rows)], dtype=np.float64)
        if np.any(np.abs(self.sigma) >= 1.0 / np.sqrt(2.0)):
            raise ValueError("cone slopes must stay below 1/sqrt(2)")
        na, nr, nd = self.n_views, self.n_rows, self.n_det
        f = self.fan
        shape = (na, nr, nd)
        rep = lambda a: np.ascontiguousarray(np.broadcast_to(a.reshape(na, 1, nd), shape).ravel())
        self.cos_r, self.sin_r, self.s_r = rep(f.cos_r), rep(f.sin_r), rep(f.s_r)
        self.row_branch = np.ascontiguousarray(rep(f.row_branch).astype(np.int32))
        src = np.array([f.source(a) for a in range(na)], dtype=np.float64)
        self.su_r = np.ascontiguousarray(np.broadcast_to(src[:, 0].reshape(na, 1, 1), shape).ravel())
        self.sv_r = np.ascontiguousarray(np.broadcast_to(src[:, 1].reshape(na, 1, 1), shape).ravel())
        self.sig_r = np.ascontiguousarray(np.broadcast_to(self.sigma.reshape(1, nr, 1), shape).ravel())

    @property
    def m(self) -> int:
        return self.n_views * self.n_rows * self.n_det

    @property
    def n(self) -> int:
        return self.N * self.N * self.Nz

    @property
    def shape(self):
        return (self.Nz, self.N, self.N)

    @property
    def sino_shape(self):
        return (self.n_views, self.n_rows, self.n_det)


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _args(g):
    return (_dp(g.cos_r), _dp(g.sin_r), _dp(g.s_r), _dp(g.su_r), _dp(g.sv_r), _dp(g.sig_r),
            g.row_branch.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))


def K(x, g: ConeGeometry) -> np.ndarray:
    """Cone-beam Joseph projection y = K x, y[a, r, t] (float64)."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(g.shape)
    y = np.empty(g.sino_shape, dtype=np.float64)
    _clib.lib().oracle_cone_forward(g.N, g.Nz, g.m, *_args(g), _dp(x), _dp(y))
    return y


def KT(y, g: ConeGeometry) -> np.ndarray:
    """Its exact transpose x = K^T y (float64, Nz x N x N)."""
    y = np.ascontiguousarray(y, dtype=np.float64).reshape(g.sino_shape)
    x = np.empty(g.shape, dtype=np.float64)
    _clib.lib().oracle_cone_transpose(g.N, g.Nz, g.m, *_args(g), _dp(y), _dp(x))
    return x


# ---------------------------------------------------------------- D in 3-D (Sec. 2 per axis)

def D(x):
    """(dx, dy, dz): dx[k,j,i] = x[k,j,i] - x[k,j,i+1], dy = x[k,j,i] - x[k,j+1,i],
    dz = x[k,j,i] - x[k+1,j,i]."""
    x = np.asarray(x, dtype=np.float64)
    return x[:, :, :-1] - x[:, :, 1:], x[:, :-1, :] - x[:, 1:, :], x[:-1, :, :] - x[1:, :, :]


def DT(dx, dy, dz):
    """Transpose of D."""
    Nz, N = dy.shape[0], dx.shape[1]
    out = np.zeros((Nz, N, N))
    out[:, :, :-1] += dx
    out[:, :, 1:] -= dx
    out[:, :-1, :] += dy
    out[:, 1:, :] -= dy
    out[:-1, :, :] += dz
    out[1:, :, :] -= dz
    return out


def H_D(N: int, Nz: int) -> np.ndarray:
    """Eigenvalues of the periodic 3-D Laplacian (eq. (f-diff) along each axis), [l, p, q]."""
    s = lambda n: np.sin(np.arange(n) * np.pi / n) ** 2
    return 4.0 * (s(Nz)[:, None, None] + s(N)[None, :, None] + s(N)[None, None, :])


def circulant_apply(x, h):
    return np.real(np.fft.ifftn(np.fft.fftn(x) * h))


def circulant_solve(r, h):
    """C^+ r with the zero-eigenvalue rule of Sec. 2."""
    hinv = np.zeros_like(h)
    nz = h != 0
    hinv[nz] = 1.0 / h[nz]
    return np.real(np.fft.ifftn(np.fft.fftn(r) * hinv))


def probe_ls(op, shape, vs) -> np.ndarray:
    """Eq. (H-fan) in least-squares form in 3-D: sum_v Re((F op(v)) conj(F v)) / sum_v |F v|^2."""
    num = np.zeros(shape)
    den = np.zeros(shape)
    for v in vs:
        Fv = np.fft.fftn(v)
        num += np.real(np.fft.fftn(op(v)) * np.conj(Fv))
        den += np.abs(Fv) ** 2
    out = np.zeros(shape)
    np.divide(num, den, out=out, where=den > 0)
    return out


def h_dc_default(g: ConeGeometry) -> float:
    one = np.ones(g.shape)
    return float(np.sum(K(one, g) ** 2) / one.size)


# ---------------------------------------------------------------- the problem and NCS

@dataclasses.dataclass
class Problem:
    """min 1/2 ||K x - b||^2 + lam TV(x) with A = [K; (beta/alpha) D] (Sec. 4.1 in 3-D)."""
    g: ConeGeometry
    b: np.ndarray
    lam: float
    alpha: float
    beta: float
    tv: str = "aniso"

    def __post_init__(self):
        self.b = np.asarray(self.b, dtype=np.float64).reshape(self.g.sino_shape)


@dataclasses.dataclass
class State:
    x: np.ndarray
    u: np.ndarray
    v: tuple


def zero_state(P: Problem) -> State:
    Nz, N = P.g.Nz, P.g.N
    return State(np.zeros(P.g.shape), np.zeros(P.g.sino_shape),
                 (np.zeros((Nz, N, N - 1)), np.zeros((Nz, N - 1, N)), np.zeros((Nz - 1, N, N))))


def A_apply(P: Problem, x):
    f = P.beta / P.alpha
    return K(x, P.g), tuple(f * d for d in D(x))


def AT_apply(P: Problem, u, v):
    return KT(u, P.g) + (P.beta / P.alpha) * DT(*v)


def AtA_apply(P: Problem, x):
    u, v = A_apply(P, x)
    return AT_apply(P, u, v)


def _pad(d, axis):
    """Difference block padded with zeros at the last index of its axis to the volume shape."""
    widths = [(0, 0)] * 3
    widths[axis] = (0, 1)
    return np.pad(d, widths)


def tv_value(P: Problem, x) -> float:
    dx, dy, dz = D(x)
    if P.tv == "aniso":
        return float(np.abs(dx).sum() + np.abs(dy).sum() + np.abs(dz).sum())
    return float(np.sqrt(_pad(dx, 2) ** 2 + _pad(dy, 1) ** 2 + _pad(dz, 0) ** 2).sum())


def objective(P: Problem, x) -> float:
    res = K(x, P.g) - P.b
    return 0.5 * float(np.sum(res * res)) + P.lam * tv_value(P, x)


def tv_dual_prox(P: Problem, z):
    """prox_{alpha g2*}: the box [-lam alpha/beta, lam alpha/beta] (anisotropic) or the
    per-voxel l2 ball of that radius over the three differences (isotropic)."""
    rad = P.lam * P.alpha / P.beta
    if P.tv == "aniso":
        return tuple(prox.clip(c, rad) for c in z)
    px, py, pz = _pad(z[0], 2), _pad(z[1], 1), _pad(z[2], 0)
    nrm = np.sqrt(px * px + py * py + pz * pz)
    fct = np.where(nrm > rad, rad / np.where(nrm > 0, nrm, 1.0), 1.0)
    return (px * fct)[:, :, :-1], (py * fct)[:, :-1, :], (pz * fct)[:-1, :, :]


def ncs_step(P: Problem, st: State, Minv) -> State:
    """Eq. (NCS): x+ = x - M^+ A^T u, xbar = 2 x+ - x, u+ = prox_{alpha g*}(u + alpha (A xbar - b))."""
    x1 = st.x - Minv(AT_apply(P, st.u, st.v))
    xb = 2.0 * x1 - st.x
    Kx, Dx = A_apply(P, xb)
    u1 = prox.prox_l2_conj(st.u + P.alpha * (Kx - P.b), P.alpha)
    v1 = tv_dual_prox(P, tuple(vc + P.alpha * dc for vc, dc in zip(st.v, Dx)))
    return State(x1, u1, v1)


def run(P: Problem, st: State, n_iter: int, Minv) -> State:
    for _ in range(n_iter):
        st = ncs_step(P, st, Minv)
    return st


def mu_probes(P: Problem, probes: int, gamma: float = 0.0) -> np.ndarray:
    """M's eigenvalues before the (A3) rescale: eq. (H-fan) over SplitMix64 probe volumes
    (seeds 1..probes) for K^T K, clamped at 0, DC entry ||K 1||^2 / ||1||^2; eq. (circ_D)
    in 3-D for D^T D."""
    g = P.g
    vs = [splitmix64_uniform(1 + q, g.n).reshape(g.shape) for q in range(probes)]
    h = np.maximum(probe_ls(lambda v: KT(K(v, g), g), g.shape, vs), 0.0)
    h[0, 0, 0] = h_dc_default(g)
    return gamma + P.alpha * h + (P.beta * P.beta / P.alpha) * H_D(g.N, g.Nz)


def a3_scaled_mu(P: Problem, mu, seed: int = 0, margin: float = 1e-2, tol: float = 1e-9, max_iter: int = 500):
    """mu <- mu rho (1 + margin), rho = lambda_max(M^{-1} alpha A^T A) by power iteration with
    the Rayleigh quotient in the M inner product (assumption (A3), Sec. 3)."""
    x = splitmix64_uniform(seed, P.g.n).reshape(P.g.shape)
    x /= np.linalg.norm(x)
    rho, old = 0.0, None
    for _ in range(max_iter):
        w = P.alpha * AtA_apply(P, x)
        rho = float(np.sum(x * w) / np.sum(x * circulant_apply(x, mu)))
        y = circulant_solve(w, mu)
        x = y / np.linalg.norm(y)
        if old is not None and abs(rho - old) <= tol * abs(rho):
            break
        old = rho
    return mu * (rho * (1.0 + margin)), rho


def dense_A(P: Problem) -> np.ndarray:
    """Dense A = [K; (beta/alpha) D_x; (beta/alpha) D_y; (beta/alpha) D_z] (small sizes)."""
    n = P.g.n
    cols = []
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        u, v = A_apply(P, e.reshape(P.g.shape))
        cols.append(np.concatenate([u.ravel()] + [c.ravel() for c in v]))
    return np.stack(cols, axis=1)


def admm_textbook(P: Problem, n_iter: int, Ad: np.ndarray):
    """ADMM on min g(Ax - b) in the textbook form of the Appendix with a dense (A^T A)^+,
    anisotropic TV: z+ = prox_{(1/alpha) g}(A x - b - lam_d), x+ = (A^T A)^+ A^T (z+ + b + lam_d),
    lam_d+ = lam_d + z+ - A x+ + b.  Returns the last x."""
    assert P.tv == "aniso"
    m = P.g.m
    a = P.alpha
    bb = np.concatenate([P.b.ravel(), np.zeros(Ad.shape[0] - m)])
    pinv = np.linalg.pinv(Ad.T @ Ad, hermitian=True)
    x = np.zeros(P.g.n)
    ld = np.zeros(Ad.shape[0])
    t = P.lam / P.beta
    for _ in range(n_iter):
        y = Ad @ x - bb - ld
        z = np.empty_like(y)
        z[:m] = y[:m] / (1.0 + 1.0 / a)
        z[m:] = prox.soft(y[m:], t)
        x = pinv @ (Ad.T @ (z + bb + ld))
        ld = ld + z - Ad @ x + bb
    return x.reshape(P.g.shape)


def lambda_max_AtA(P: Problem, seed: int = 0, tol: float = 1e-9, max_iter: int = 500) -> float:
    """lambda_max(A^T A) by power iteration with the Rayleigh quotient (SplitMix64 start)."""
    x = splitmix64_uniform(seed, P.g.n).reshape(P.g.shape)
    x /= np.linalg.norm(x)
    lm, old = 0.0, None
    for _ in range(max_iter):
        w = AtA_apply(P, x)
        lm = float(np.sum(x * w))
        x = w / np.linalg.norm(w)
        if old is not None and abs(lm - old) <= tol * abs(lm):
            break
        old = lm
    return lm


def pdhg_gamma(P: Problem, margin: float = 1e-2) -> float:
    """gamma_P = alpha lambda_max(A^T A) (1 + margin): the step condition of eq. (PDHG)."""
    return P.alpha * lambda_max_AtA(P) * (1.0 + margin)


def pdhg_step(P: Problem, st: State, gamma_p: float) -> State:
    """Eq. (PDHG): x+ = x - gamma_P^{-1} A^T u, then NCS's dual update (M = gamma_P I)."""
    return ncs_step(P, st, lambda r: r / gamma_p)
