"""Pins of the oracle's circulant part: eq. (f-diff) against a dense
eigendecomposition, the FFT solve against a dense DFT built from its
definition, the pseudo-inverse rule of Sec. 2, eq. (circ_D) as the spectrum of
the periodic 2-D Laplacian, and the probe estimator of eq. (H-fan)."""
import math

import numpy as np
import pytest

from oracle import circulant as ci
from oracle import operators as op


def dft_matrix(n):
    p = np.arange(n)
    return np.exp(-2j * math.pi * np.outer(p, p) / n)


@pytest.mark.parametrize("n", [5, 8, 16])
def test_ltilde_eigenvalues(n):
    ev = np.sort(np.linalg.eigvalsh(ci.Ltilde_matrix(n)))
    assert np.allclose(ev, np.sort(ci.ltilde_eigs(n)), atol=1e-12)
    # and the DFT basis diagonalises it with exactly those eigenvalues, in order
    F = dft_matrix(n)
    Dg = F @ ci.Ltilde_matrix(n) @ np.linalg.inv(F)
    assert np.allclose(np.diag(Dg).real, ci.ltilde_eigs(n), atol=1e-12)
    assert np.max(np.abs(Dg - np.diag(np.diag(Dg)))) < 1e-12


def test_H_D_is_spectrum_of_periodic_2d_laplacian():
    N = 16
    Lt = ci.Ltilde_matrix(N)
    P = np.kron(np.eye(N), Lt) + np.kron(Lt, np.eye(N))
    ev = np.sort(np.linalg.eigvalsh(P))
    assert np.allclose(ev, np.sort(ci.H_D(N).ravel()), atol=1e-11)
    x = np.random.default_rng(0).standard_normal((N, N))
    assert np.allclose(ci.circulant_apply(x, ci.H_D(N)).ravel(), P @ x.ravel(), atol=1e-12)


def test_circulant_solve_against_dense_dft():
    N = 16
    F2 = np.kron(dft_matrix(N), dft_matrix(N))
    rng = np.random.default_rng(1)
    h = rng.uniform(0.5, 3.0, size=(N, N))
    h = 0.5 * (h + h[(-np.arange(N)) % N][:, (-np.arange(N)) % N])   # real circulant -> symmetric spectrum
    dense = np.linalg.inv(F2) @ np.diag(1.0 / h.ravel()) @ F2
    assert np.max(np.abs(dense.imag)) < 1e-12
    r = rng.standard_normal((N, N))
    assert np.allclose(ci.circulant_solve(r, h).ravel(), dense.real @ r.ravel(), atol=1e-12)
    # C C^+ = I when h has no zeros
    assert np.allclose(ci.circulant_apply(ci.circulant_solve(r, h), h), r, atol=1e-12)


def test_pseudo_inverse_rule_zero_entries():
    N = 8
    h = ci.H_D(N)                      # h[0,0] = 0: the constant image is in the null space
    r = np.random.default_rng(2).standard_normal((N, N))
    z = ci.circulant_solve(r, h)
    assert abs(z.sum()) < 1e-12         # DC component mapped to 0
    Lt = ci.Ltilde_matrix(N)
    P = np.kron(np.eye(N), Lt) + np.kron(Lt, np.eye(N))
    assert np.allclose(z.ravel(), np.linalg.pinv(P, hermitian=True) @ r.ravel(), atol=1e-11)


def test_H_R_shape():
    N = 12
    H = ci.H_R(N, 3.0, 7.0)
    assert H[0, 0] == 7.0
    assert H[0, 1] == pytest.approx(3.0) and H[1, 1] == pytest.approx(3.0 / math.sqrt(2))
    assert H[0, N - 1] == H[0, 1] and H[5, 7] == H[7, 5] == H[N - 5, N - 7]


def test_probe_ratio_recovers_exact_circulant():
    N = 16
    rng = np.random.default_rng(3)
    h = ci.H_D(N) + 1.0
    vs = [rng.standard_normal((N, N)) for _ in range(2)]
    est = ci.probe_ratio(lambda v: ci.circulant_apply(v, h), N, vs)
    assert np.allclose(est, h, atol=1e-10)


def test_C_R_default_matches_probe_at_low_frequency():
    """The default C_R = n_angles N / pi reproduces the probe-estimated spectrum
    of K^T K (eq. (H-fan)) at the lowest nonzero frequencies within 25%."""
    N, na, nd = 64, 90, 92
    g = op.Geometry(N, na, nd)
    rng = np.random.default_rng(4)
    vs = [rng.standard_normal((N, N)) for _ in range(16)]
    h = ci.probe_ratio(lambda v: op.KT(op.K(v, g), g), N, vs)
    j = np.arange(N)
    jp = np.minimum(j, N - j)
    r = np.sqrt(jp[:, None] ** 2 + jp[None, :] ** 2)
    sel = (r > 0.5) & (r < 4.5)
    ratio = np.mean(h[sel] * r[sel]) / ci.c_r_default(g)
    assert 0.75 < ratio < 1.25


def test_h_dc_default_is_rayleigh_quotient():
    g = op.Geometry(16, 12, 24)
    one = np.ones((16, 16))
    KtK1 = op.KT(op.K(one, g), g)
    assert ci.h_dc_default(g) == pytest.approx(np.sum(one * KtK1) / 256.0, rel=1e-12)


def test_probe_ls_recovers_circulant_eigenvalues_and_matches_one_probe_ratio():
    """Eq. (H-fan), least-squares form: for a circulant operator it returns the exact
    eigenvalues whatever the probes; with a single probe it is the real part of the
    paper's ratio."""
    N = 12
    rng = np.random.default_rng(4)
    h = rng.uniform(0.5, 3.0, (N, N))
    h = 0.5 * (h + np.roll(np.flip(h), 1, axis=(0, 1)))      # h(-j, -k) = h(j, k): a real operator
    op = lambda v: ci.circulant_apply(v, h)
    vs = [rng.standard_normal((N, N)) for _ in range(3)]
    assert np.max(np.abs(ci.probe_ls(op, N, vs) - h)) <= 1e-12 * h.max()
    one = ci.probe_ls(op, N, vs[:1])
    assert np.max(np.abs(one - np.real(ci.probe_ratio(op, N, vs[:1])))) <= 1e-12 * h.max()
