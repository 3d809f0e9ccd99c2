"""FP64 oracle for the circulant matrix M and its FFT solve.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 2: a circulant C = F^{-1} diag(h) F has C^+ = F^{-1} diag(h)^+ F where
diag(h)^+ inverts the nonzero entries and keeps the zeros.  Eq. (f-diff): the
periodic 1-D Laplacian L~_n has eigenvalues d_{i+1} = 4 sin^2(i pi / n).
Sec. 4.1.1, eqs. (circ_R), (circ_D): R^T R ~ F^{-1} diag(h_R) F with
H_R[j,k] = C_R / sqrt(min(j,N-j)^2 + min(k,N-k)^2) except at j=k=0 (the DC
entry, tuned separately), and D^T D ~ F^{-1} diag(h_D) F with
H_D[j,k] = 4 (sin^2(j pi/N) + sin^2(k pi/N)).

Readings where the paper is silent (each listed in the design notes):
  * M's eigenvalues mu = gamma + alpha*H_R + (beta^2/alpha)*H_D (+ alpha*kappa^2
    for the PET nonnegativity row), i.e. M = gamma I + alpha C with
    C ~ A^T A for A = [K; (beta/alpha) D; kappa I];
  * C_R defaults to n_angles * N / pi;
  * the DC entry of H_R defaults to ||K 1||^2 / ||1||^2.
"""
from __future__ import annotations

import math

import numpy as np

from .operators import Geometry, K


def Ltilde_matrix(n: int) -> np.ndarray:
    """Dense periodic Laplacian L~_n of Sec. 2 (2 on the diagonal, -1 on the
    two neighbours, cyclically)."""
    L = 2.0 * np.eye(n)
    for i in range(n):
        L[i, (i + 1) % n] = -1.0
        L[i, (i - 1) % n] = -1.0
    return L


def ltilde_eigs(n: int) -> np.ndarray:
    """Eq. (f-diff): d_{i+1} = 4 sin^2(i pi / n), i = 0..n-1."""
    i = np.arange(n, dtype=np.float64)
    return 4.0 * np.sin(i * math.pi / n) ** 2


def H_D(N: int) -> np.ndarray:
    """Eq. (circ_D)."""
    j = np.arange(N, dtype=np.float64)
    s2 = np.sin(j * math.pi / N) ** 2
    return 4.0 * (s2[:, None] + s2[None, :])


def H_R(N: int, c_r: float, h_dc: float) -> np.ndarray:
    """Eq. (circ_R) with the DC entry set to h_dc."""
    j = np.arange(N)
    jp = np.minimum(j, N - j).astype(np.float64)
    r2 = jp[:, None] ** 2 + jp[None, :] ** 2
    r2[0, 0] = 1.0
    H = c_r / np.sqrt(r2)
    H[0, 0] = h_dc
    return H


def c_r_default(g: Geometry) -> float:
    """n_angles * N / pi: backprojection sums n_angles angles in place of the
    integral over [0, pi), and the transform of 1/|r| is 1/|nu| with nu = j'/N."""
    return g.n_angles * g.N / math.pi


def h_dc_default(g: Geometry) -> float:
    """Rayleigh quotient of K^T K on the constant image, (F K^T K F^{-1})_{00}."""
    one = np.ones((g.N, g.N))
    return float(np.sum(K(one, g) ** 2) / one.size)


def mu_table(g: Geometry, alpha: float, beta: float, gamma: float,
             c_r: float | None = None, h_dc: float | None = None, kappa: float = 0.0) -> np.ndarray:
    """Eigenvalues of M = gamma I + alpha C (N x N, float64), before any A3 rescale."""
    c_r = c_r_default(g) if c_r is None else c_r
    h_dc = h_dc_default(g) if h_dc is None else h_dc
    N = g.N
    return gamma + alpha * H_R(N, c_r, h_dc) + (beta * beta / alpha) * H_D(N) + alpha * kappa * kappa


def circulant_apply(x: np.ndarray, h: np.ndarray) -> np.ndarray:
    """C x = F^{-1} diag(h) F x for a real image x."""
    return np.real(np.fft.ifft2(np.fft.fft2(x) * h))


def circulant_solve(r: np.ndarray, h: np.ndarray) -> np.ndarray:
    """C^+ r = F^{-1} diag(h)^+ F r (Sec. 2), entries h == 0 map to 0."""
    hinv = np.zeros_like(h)
    nz = h != 0
    hinv[nz] = 1.0 / h[nz]
    return np.real(np.fft.ifft2(np.fft.fft2(r) * hinv))


def probe_ls(op, N: int, vs) -> np.ndarray:
    """Eq. (H-fan) in least-squares form: sum over probe images v of
    Re((F op(v)) conj(F v)) divided by sum of |F v|^2 (0 where every F v vanishes).
    For one probe it equals the real part of probe_ratio; for a circulant op it is the
    op's eigenvalues for any probes."""
    num = np.zeros((N, N))
    den = np.zeros((N, N))
    for v in vs:
        Fv = np.fft.fft2(v)
        Fw = np.fft.fft2(op(v))
        num += np.real(Fw * np.conj(Fv))
        den += np.abs(Fv) ** 2
    out = np.zeros((N, N))
    np.divide(num, den, out=out, where=den > 0)
    return out


def probe_ratio(op, N: int, vs) -> np.ndarray:
    """Eq. (H-fan): the average over probe images v of (F op(v))_i / (F v)_i,
    an estimate of the circulant eigenvalues of a near-circulant op."""
    acc = np.zeros((N, N), dtype=np.complex128)
    for v in vs:
        Fv = np.fft.fft2(v)
        acc += np.fft.fft2(op(v)) / Fv
    return np.real(acc / len(vs))
