"""FP64 oracle for the solvers: NCS (Sec. 1.2, eq. (NCS); Sec. 4), PDHG (eq.
(PDHG)), dense ADMM (eq. (ADMM) and the textbook form of the Appendix), the
objective, and the power iterations behind assumption (A3).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The problem is min g(Ax - b) with A = [K; (beta/alpha) D; kappa I]
(Sec. 4.1 for CT, Sec. 4.2 for PET with the nonnegativity row of its remark).
CT:  g(y, z) = 1/2 ||y||^2 + (lam alpha/beta) TV-norm(z)       (kappa = 0)
PET: g(y, z, s) = sum_i l(y_i + r_i; b_i) + (lam alpha/beta)||z||_1 + delta_{R+}(s)
The dual iterate is (u, vh, vv, s) for the rows (K, D_h, D_v, I).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import prox
from .circulant import circulant_apply, circulant_solve
from .operators import D, DT, Geometry, K, KT, D1_matrix


@dataclasses.dataclass
class Problem:
    g: Geometry
    b: np.ndarray                 # CT: measured sinogram; PET: counts y
    lam: float
    alpha: float
    beta: float
    kind: str = "ct"              # "ct" | "pet"
    tv: str = "aniso"             # "aniso" | "iso"
    kappa: float = 0.0            # weight of the nonnegativity row (PET)
    r_bg: np.ndarray | None = None  # PET background (sinogram-shaped)

    def __post_init__(self):
        self.b = np.asarray(self.b, dtype=np.float64).reshape(self.g.n_angles, self.g.n_det)
        if self.r_bg is not None:
            self.r_bg = np.asarray(self.r_bg, dtype=np.float64).reshape(self.b.shape)


@dataclasses.dataclass
class State:
    x: np.ndarray
    u: np.ndarray
    vh: np.ndarray
    vv: np.ndarray
    s: np.ndarray | None = None

    def copy(self):
        return State(self.x.copy(), self.u.copy(), self.vh.copy(), self.vv.copy(),
                     None if self.s is None else self.s.copy())


def zero_state(P: Problem) -> State:
    N = P.g.N
    return State(np.zeros((N, N)), np.zeros_like(P.b), np.zeros((N, N - 1)), np.zeros((N - 1, N)),
                 np.zeros((N, N)) if P.kappa != 0.0 else None)


# ---------------------------------------------------------------- A and A^T

def A_apply(P: Problem, x):
    """A x = (K x, (beta/alpha) D_h x, (beta/alpha) D_v x, kappa x)."""
    dh, dv = D(x)
    f = P.beta / P.alpha
    return K(x, P.g), f * dh, f * dv, (P.kappa * x if P.kappa != 0.0 else None)


def AT_apply(P: Problem, u, vh, vv, s=None):
    """A^T (u, vh, vv, s) = K^T u + (beta/alpha) D^T (vh, vv) + kappa s."""
    r = KT(u, P.g) + (P.beta / P.alpha) * DT(vh, vv)
    if s is not None and P.kappa != 0.0:
        r = r + P.kappa * s
    return r


def AtA_apply(P: Problem, x):
    Ax = A_apply(P, x)
    return AT_apply(P, *Ax)


# ---------------------------------------------------------------- prox of alpha g*

def _pad_h(dh):
    N = dh.shape[0]
    out = np.zeros((N, N))
    out[:, :-1] = dh
    return out


def _pad_v(dv):
    N = dv.shape[1]
    out = np.zeros((N, N))
    out[:-1, :] = dv
    return out


def tv_dual_prox(P: Problem, zh, zv):
    """prox_{alpha g2*} of the TV block: the box [-lam alpha/beta, lam alpha/beta]
    (Sec. 4.1, anisotropic) or the per-pixel l2 ball of that radius (isotropic)."""
    rad = P.lam * P.alpha / P.beta
    if P.tv == "aniso":
        return prox.clip(zh, rad), prox.clip(zv, rad)
    ph, pv = prox.ball2(_pad_h(zh), _pad_v(zv), rad)
    return ph[:, :-1], pv[:-1, :]


def data_dual_prox(P: Problem, u, Kxb):
    """prox_{alpha g1*}(u + alpha (K xbar - b)) for CT; S(u + alpha (K xbar + r); alpha b)
    for PET (Sec. 4.2, background read as g1(y) = l(y + r; b))."""
    a = P.alpha
    if P.kind == "ct":
        return prox.prox_l2_conj(u + a * (Kxb - P.b), a)
    r = P.r_bg if P.r_bg is not None else 0.0
    return prox.S_kl(u + a * (Kxb + r), a * P.b)


# ---------------------------------------------------------------- objective

def tv_value(P: Problem, x) -> float:
    dh, dv = D(x)
    if P.tv == "aniso":
        return float(np.abs(dh).sum() + np.abs(dv).sum())
    return float(np.sqrt(_pad_h(dh) ** 2 + _pad_v(dv) ** 2).sum())


def kl_value(y, mu) -> float:
    """sum_i mu_i - y_i + y_i log(y_i / mu_i), with 0 log 0 = 0."""
    y = np.asarray(y, dtype=np.float64)
    mu = np.asarray(mu, dtype=np.float64)
    pos = y > 0
    val = np.sum(mu - y)
    val += np.sum(y[pos] * np.log(y[pos] / mu[pos]))
    return float(val)


def objective(P: Problem, x) -> float:
    """CT: 1/2 ||K x - b||^2 + lam TV(x) (Sec. 4.1).  PET: KL(b, K x+ + r) +
    lam TV(x+) at x+ = max(x, 0), the feasible point nearest x (Sec. 4.2)."""
    x = np.asarray(x, dtype=np.float64)
    if P.kind == "ct":
        res = K(x, P.g) - P.b
        return 0.5 * float(np.sum(res * res)) + P.lam * tv_value(P, x)
    xp = np.maximum(x, 0.0)
    r = P.r_bg if P.r_bg is not None else 0.0
    return kl_value(P.b, K(xp, P.g) + r) + P.lam * tv_value(P, xp)


# ---------------------------------------------------------------- iterations

def ncs_step(P: Problem, st: State, Minv) -> State:
    """One NCS iteration (eq. (NCS); explicit forms of Sec. 4.1 / 4.2):
    x+ = x - M^+ A^T u;  xbar = 2 x+ - x;  each dual block u+ = prox_{alpha g*}(u + alpha (A xbar - b))."""
    r = AT_apply(P, st.u, st.vh, st.vv, st.s)
    x1 = st.x - Minv(r)
    xb = 2.0 * x1 - st.x
    u1 = data_dual_prox(P, st.u, K(xb, P.g))
    dh, dv = D(xb)
    vh1, vv1 = tv_dual_prox(P, st.vh + P.beta * dh, st.vv + P.beta * dv)
    s1 = None
    if st.s is not None:
        s1 = prox.min0(st.s + P.alpha * P.kappa * xb)
    return State(x1, u1, vh1, vv1, s1)


def pdhg_step(P: Problem, st: State, gamma_p: float) -> State:
    """One PDHG iteration (eq. (PDHG)): x+ = x - gamma^{-1} A^T u, then the same
    dual update as NCS."""
    return ncs_step(P, st, lambda r: r / gamma_p)


def run(P: Problem, st: State, n_iter: int, Minv, record=None) -> State:
    for k in range(n_iter):
        st = ncs_step(P, st, Minv)
        if record is not None:
            record(k, st)
    return st


def circulant_Minv(mu):
    return lambda r: circulant_solve(r, mu)


# ---------------------------------------------------------------- dense ADMM (tiny sizes)

def dense_A(P: Problem) -> np.ndarray:
    """Dense A = [K; (beta/alpha) (I (x) D_n); (beta/alpha) (D_n (x) I); kappa I]."""
    N = P.g.N
    n = N * N
    Kd = np.zeros((P.g.m, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        Kd[:, k] = K(e.reshape(N, N), P.g).ravel()
    Dn = D1_matrix(N)
    f = P.beta / P.alpha
    blocks = [Kd, f * np.kron(np.eye(N), Dn), f * np.kron(Dn, np.eye(N))]
    if P.kappa != 0.0:
        blocks.append(P.kappa * np.eye(n))
    return np.vstack(blocks)


def _split(P: Problem, w):
    N = P.g.N
    m = P.g.m
    u = w[:m].reshape(P.g.n_angles, P.g.n_det)
    vh = w[m:m + N * (N - 1)].reshape(N, N - 1)
    vv = w[m + N * (N - 1):m + 2 * N * (N - 1)].reshape(N - 1, N)
    return u, vh, vv


def admm_textbook(P: Problem, n_iter: int, Ad: np.ndarray, x0=None, lam0=None, record=None):
    """ADMM applied to min g(Ax - b) in its textbook (z, x, lambda) form
    (Appendix, "Derivation from ADMM"), CT only, with a dense pseudo-inverse:
      z+ = prox_{(1/alpha) g}(A x - b - lambda)
      x+ = (A^T A)^+ A^T (z+ + b + lambda)
      lambda+ = lambda + z+ - A x+ + b
    Returns the list of x iterates x^1..x^n."""
    assert P.kind == "ct"
    N = P.g.N
    n = N * N
    a = P.alpha
    bb = np.concatenate([P.b.ravel(), np.zeros(Ad.shape[0] - P.g.m)])
    AtA_pinv = np.linalg.pinv(Ad.T @ Ad, hermitian=True)
    x = np.zeros(n) if x0 is None else np.ravel(x0).copy()
    lam = np.zeros(Ad.shape[0]) if lam0 is None else lam0.copy()
    xs = []
    for k in range(n_iter):
        w = Ad @ x - bb - lam
        u, zh, zv = _split(P, w)
        z_data = u / (1.0 + 1.0 / a)                   # prox of (1/alpha) * 1/2||.||^2
        t = P.lam / P.beta                              # (1/alpha) * lam alpha / beta
        if P.tv == "aniso":
            zh1, zv1 = prox.soft(zh, t), prox.soft(zv, t)
        else:
            ph, pv = prox.soft_iso(_pad_h(zh), _pad_v(zv), t)
            zh1, zv1 = ph[:, :-1], pv[:-1, :]
        z = np.concatenate([z_data.ravel(), zh1.ravel(), zv1.ravel()])
        x = AtA_pinv @ (Ad.T @ (z + bb + lam))
        lam = lam + z - Ad @ x + bb
        xs.append(x.reshape(N, N).copy())
        if record is not None:
            record(k, x)
    return xs


def explicit_inverse(AtA: np.ndarray) -> np.ndarray:
    """(A^T A)^+ as an explicit dense matrix: the inverse through a Cholesky factor when
    A^T A is positive definite, else the eigendecomposition pseudo-inverse (Sec. 2)."""
    import scipy.linalg as sla
    n = AtA.shape[0]
    try:
        c = sla.cho_factor(AtA, check_finite=False)
        return sla.cho_solve(c, np.eye(n), check_finite=False)
    except np.linalg.LinAlgError:
        return np.linalg.pinv(AtA, hermitian=True)


def admm_explicit(P: Problem, n_iter: int, AtA_inv: np.ndarray, x0=None, record=None):
    """The textbook ADMM of admm_textbook (Appendix, "Derivation from ADMM"), CT only, with
    A applied as the operators K and D (A = [K; (beta/alpha) D]) and the x-update through
    an explicit dense (A^T A)^+:
      z+ = prox_{(1/alpha) g}(A x - b - lambda)
      x+ = (A^T A)^+ A^T (z+ + b + lambda)
      lambda+ = lambda + z+ - A x+ + b
    Returns the list of x iterates x^1..x^n (record(k, x) is called on each)."""
    assert P.kind == "ct"
    N = P.g.N
    a = P.alpha
    f = P.beta / P.alpha
    x = np.zeros((N, N)) if x0 is None else np.array(x0, dtype=np.float64).reshape(N, N)
    lu = np.zeros_like(P.b)
    lh = np.zeros((N, N - 1))
    lv = np.zeros((N - 1, N))
    Kx = K(x, P.g)
    dh, dv = D(x)
    xs = []
    for k in range(n_iter):
        zu = (Kx - P.b - lu) / (1.0 + 1.0 / a)           # prox of (1/alpha) * 1/2||.||^2
        t = P.lam / P.beta                                # (1/alpha) * lam alpha / beta
        wh, wv = f * dh - lh, f * dv - lv
        if P.tv == "aniso":
            zh, zv = prox.soft(wh, t), prox.soft(wv, t)
        else:
            ph, pv = prox.soft_iso(_pad_h(wh), _pad_v(wv), t)
            zh, zv = ph[:, :-1], pv[:-1, :]
        rhs = KT(zu + P.b + lu, P.g) + f * DT(zh + lh, zv + lv)
        x = (AtA_inv @ rhs.ravel()).reshape(N, N)
        Kx = K(x, P.g)
        dh, dv = D(x)
        lu = lu + zu - Kx + P.b
        lh = lh + zh - f * dh
        lv = lv + zv - f * dv
        xs.append(x.copy())
        if record is not None:
            record(k, x)
    return xs


def admm_pcg(P: Problem, n_iter: int, n_cg: int, Minv, x0=None, record=None):
    """ADMM in the textbook form of admm_textbook (Appendix, "Derivation from ADMM"),
    CT only, with the x-update (A^T A) x = A^T (z+ + b + lambda) solved approximately
    by n_cg steps of conjugate gradients preconditioned by the circulant M (Sec. 1.3,
    the PCG inner loop of the ADMM comparator) and started from the current x.
    Returns the list of x iterates x^1..x^n."""
    assert P.kind == "ct"
    N = P.g.N
    f = P.beta / P.alpha
    a = P.alpha
    x = np.zeros((N, N)) if x0 is None else np.array(x0, dtype=np.float64).reshape(N, N)
    lu = np.zeros_like(P.b)
    lh = np.zeros((N, N - 1))
    lv = np.zeros((N - 1, N))

    def AtA(v):
        dh, dv = D(v)
        return KT(K(v, P.g), P.g) + f * f * DT(dh, dv)

    Kx = K(x, P.g)
    dh, dv = D(x)
    xs = []
    for k in range(n_iter):
        # z+ = prox_{(1/alpha) g}(A x - b - lambda)
        zu = (Kx - P.b - lu) / (1.0 + 1.0 / a)
        t = P.lam / P.beta
        wh, wv = f * dh - lh, f * dv - lv
        if P.tv == "aniso":
            zh, zv = prox.soft(wh, t), prox.soft(wv, t)
        else:
            ph, pv = prox.soft_iso(_pad_h(wh), _pad_v(wv), t)
            zh, zv = ph[:, :-1], pv[:-1, :]
        # x+ ~ (A^T A)^{-1} A^T (z+ + b + lambda) by PCG from x
        rhs = KT(zu + P.b + lu, P.g) + f * DT(zh + lh, zv + lv)
        r = rhs - AtA(x)
        sv = Minv(r)
        pv_ = sv.copy()
        rs = float(np.sum(r * sv))
        for _ in range(n_cg):
            if rs <= 0.0:
                break
            q = AtA(pv_)
            step = rs / float(np.sum(pv_ * q))
            x = x + step * pv_
            r = r - step * q
            sv = Minv(r)
            rs_new = float(np.sum(r * sv))
            pv_ = sv + (rs_new / rs) * pv_
            rs = rs_new
        # lambda+ = lambda + z+ - A x+ + b
        Kx = K(x, P.g)
        dh, dv = D(x)
        lu = lu + zu - Kx + P.b
        lh = lh + zh - f * dh
        lv = lv + zv - f * dv
        xs.append(x.copy())
        if record is not None:
            record(k, x)
    return xs


def dense_Minv(Md: np.ndarray):
    """M^+ for a dense symmetric M (pseudo-inverse through its eigendecomposition)."""
    Mp = np.linalg.pinv(Md, hermitian=True)
    return lambda r: (Mp @ np.ravel(r)).reshape(r.shape)


# ---------------------------------------------------------------- seminorm of Sec. 3.2

def seminorm_sq(P: Problem, Mapply, dx, du, dvh, dvv, ds=None) -> float:
    """D^2(x, u) = ||u - alpha A x||^2 + x^T (alpha M - alpha^2 A^T A) x (Sec. 3.2)."""
    a = P.alpha
    Ax = A_apply(P, dx)
    acc = float(np.sum((du - a * Ax[0]) ** 2) + np.sum((dvh - a * Ax[1]) ** 2)
                + np.sum((dvv - a * Ax[2]) ** 2))
    Ax2 = float(np.sum(Ax[0] ** 2) + np.sum(Ax[1] ** 2) + np.sum(Ax[2] ** 2))
    if ds is not None and Ax[3] is not None:
        acc += float(np.sum((ds - a * Ax[3]) ** 2))
        Ax2 += float(np.sum(Ax[3] ** 2))
    return acc + a * float(np.sum(dx * Mapply(dx))) - a * a * Ax2


# ---------------------------------------------------------------- power iterations (A3)

_SM_GOLD = 0x9E3779B97F4A7C15
_SM_M1 = 0xBF58476D1CE4E5B9
_SM_M2 = 0x94D049BB133111EB
_U64 = (1 << 64) - 1


def splitmix64_uniform(seed: int, count: int) -> np.ndarray:
    """Counter-based uniforms in [-1, 1): element k is SplitMix64 (Steele, Lea,
    Flood 2014) applied to the state seed + (k+1)*0x9E3779B97F4A7C15, top 53
    bits scaled to [0, 1), then mapped to 2u - 1."""
    k = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _U64) + k * np.uint64(_SM_GOLD)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(_SM_M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(_SM_M2)
        z = z ^ (z >> np.uint64(31))
    u = (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return 2.0 * u - 1.0


def power_rho(P: Problem, mu: np.ndarray, x0: np.ndarray, tol: float = 1e-9, max_iter: int = 500):
    """rho = lambda_max(M^{-1} alpha A^T A) by power iteration: x <- M^{-1} alpha A^T A x,
    normalised, with the Rayleigh quotient in the M inner product,
    <x, alpha A^T A x> / <x, M x>.  Stops at relative change < tol.
    Returns (rho, iterations)."""
    x = x0 / np.linalg.norm(x0)
    rho_old = None
    it = 0
    for it in range(1, max_iter + 1):
        w = P.alpha * AtA_apply(P, x)
        rho = float(np.sum(x * w) / np.sum(x * circulant_apply(x, mu)))
        y = circulant_solve(w, mu)
        x = y / np.linalg.norm(y)
        if rho_old is not None and abs(rho - rho_old) <= tol * abs(rho):
            break
        rho_old = rho
    return rho, it


def power_lmax_AtA(P: Problem, x0: np.ndarray, tol: float = 1e-9, max_iter: int = 500):
    """lambda_max(A^T A) by power iteration with the Rayleigh quotient
    <x, A^T A x>/<x, x> (for PDHG's gamma/alpha >= lambda_max, eq. (PDHG))."""
    x = x0 / np.linalg.norm(x0)
    lm_old = None
    it = 0
    for it in range(1, max_iter + 1):
        w = AtA_apply(P, x)
        lm = float(np.sum(x * w) / np.sum(x * x))
        x = w / np.linalg.norm(w)
        if lm_old is not None and abs(lm - lm_old) <= tol * abs(lm):
            break
        lm_old = lm
    return lm, it


def a3_scaled_mu(P: Problem, mu: np.ndarray, seed: int = 0, margin: float = 1e-2,
                 tol: float = 1e-9, max_iter: int = 500):
    """Rescale M so that (A3) M >= alpha A^T A holds with a margin: mu <- mu * rho * (1 + margin)
    with rho = lambda_max(M^{-1} alpha A^T A) (reading: the paper tunes M by hand and
    never checks (A3)).  Returns (mu_scaled, rho)."""
    x0 = splitmix64_uniform(seed, P.g.n).reshape(P.g.N, P.g.N)
    rho, _ = power_rho(P, mu, x0, tol=tol, max_iter=max_iter)
    return mu * (rho * (1.0 + margin)), rho


def pdhg_gamma(P: Problem, seed: int = 0, margin: float = 1e-2, tol: float = 1e-9, max_iter: int = 500):
    """gamma_P = alpha * lambda_max(A^T A) * (1 + margin) (eq. (PDHG) condition)."""
    x0 = splitmix64_uniform(seed, P.g.n).reshape(P.g.N, P.g.N)
    lm, _ = power_lmax_AtA(P, x0, tol=tol, max_iter=max_iter)
    return P.alpha * lm * (1.0 + margin), lm
