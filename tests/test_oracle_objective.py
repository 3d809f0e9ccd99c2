"""Pins of the oracle's objective (Sec. 4.1: 1/2||Kx - b||^2 + lam TV(x); Sec. 4.2:
KL(b, Kx + r) + lam TV(x) at x+ = max(x, 0)) and of the eigenvalues of M
(M = gamma I + alpha C with C ~ A^T A, A = [K; (beta/alpha) D; kappa I]; eqs.
(circ_R), (circ_D)), against values worked out by hand and dense operators built
from their definitions.

The hand-worked case: a 3 x 3 image seen at the one angle theta = 0 by 3 bins at
unit spacing.  The bins then sit on the pixel-centre columns, so K x is the vector of
column sums (Joseph weights 1/|cos 0| = 1, no interpolation)."""
import math

import numpy as np
import pytest

from oracle import circulant as ci
from oracle import operators as op
from oracle import solvers as so
import synth
from helpers import oproj

X3 = np.array([[1.0, 2.0, 4.0],
               [0.0, 3.0, 1.0],
               [2.0, 2.0, 5.0]])
B3 = np.array([[1.0, 2.0, 3.0]])          # one angle, three bins


def _p3(tv, kind="ct", b=B3, r_bg=None):
    g = op.Geometry(3, 1, 3)
    return so.Problem(g, b, lam=0.5, alpha=1.0, beta=1.0, tv=tv, kind=kind, kappa=1.0 if kind == "pet" else 0.0,
                      r_bg=r_bg)


def test_column_sums_at_theta_zero():
    assert np.array_equal(op.K(X3, op.Geometry(3, 1, 3)), np.array([[3.0, 7.0, 10.0]]))


def test_ct_objective_by_hand():
    # residual (3, 7, 10) - (1, 2, 3) = (2, 5, 7): 1/2 (4 + 25 + 49) = 39
    # horizontal differences x[j][i] - x[j][i+1]: (-1, -2), (-3, 2), (0, -3)
    # vertical differences x[j][i] - x[j+1][i]: (1, -1, 3), (-2, 1, -4)
    # anisotropic TV: the absolute horizontal differences sum to 11, the vertical ones to 12
    assert so.tv_value(_p3("aniso"), X3) == 23.0
    assert so.objective(_p3("aniso"), X3) == 39.0 + 0.5 * 23.0
    # isotropic TV: per pixel sqrt(dh^2 + dv^2), dh = 0 in the last column, dv = 0 in the last row
    # (0,0) (-1, 1); (0,1) (-2,-1); (0,2) (0, 3); (1,0) (-3,-2); (1,1) (2, 1); (1,2) (0,-4);
    # (2,0) (0, 0); (2,1) (-3, 0); (2,2) (0, 0)
    iso = math.sqrt(2) + math.sqrt(5) + 3 + math.sqrt(13) + math.sqrt(5) + 4 + 0 + 3 + 0
    assert so.tv_value(_p3("iso"), X3) == pytest.approx(iso, rel=1e-15)
    assert so.objective(_p3("iso"), X3) == pytest.approx(39.0 + 0.5 * iso, rel=1e-15)


def test_pet_objective_by_hand():
    # x+ = max(x, 0) clamps the one negative pixel; counts y = (2, 0, 9), background r = 1:
    # mu = K x+ + r = (3 + 1, 7 + 1, 10 + 1) with x[1][0] = -1 -> 0 leaving column 0 at 3
    x = X3.copy()
    x[1, 0] = -1.0
    y = np.array([[2.0, 0.0, 9.0]])
    r = np.ones((1, 3))
    mu = np.array([4.0, 8.0, 11.0])
    kl = (4 - 2 + 2 * math.log(2 / 4)) + (8 - 0) + (11 - 9 + 9 * math.log(9 / 11))
    P = _p3("aniso", kind="pet", b=y, r_bg=r)
    assert so.kl_value(y, mu.reshape(1, 3)) == pytest.approx(kl, rel=1e-15)
    assert so.objective(P, x) == pytest.approx(kl + 0.5 * 23.0, rel=1e-15)


N, NA, ND = 16, 24, 26


@pytest.mark.parametrize("tv", ["aniso", "iso"])
def test_dense_admm_minimiser_minimises_the_objective(tv):
    """The dense-inverse ADMM of the Appendix (its z-update uses the prox of lam TV, not the
    objective) converges to a point that the objective cannot improve: no decrease along
    +-x* (where TV is homogeneous, so a wrong lam factor or TV norm shows at first order) or
    along random directions."""
    pr = synth.ct_problem(0, N, NA, ND, 5, 0.01, oproj(N, NA, ND))
    g = op.Geometry(N, NA, ND)
    P = so.Problem(g, pr["b"], lam=0.5, alpha=10.0, beta=10.0, tv=tv)
    xs = so.admm_textbook(P, 2500, so.dense_A(P))
    xstar = xs[-1]
    f = so.objective(P, xstar)
    rng = np.random.default_rng(4)
    dirs = [xstar / np.linalg.norm(xstar), -xstar / np.linalg.norm(xstar)]
    dirs += [d / np.linalg.norm(d) for d in rng.standard_normal((6, N, N))]
    for d in dirs:
        for eps in (1e-2, 1e-3):
            assert so.objective(P, xstar + eps * np.linalg.norm(xstar) * d) >= f * (1 - 1e-12)
    # and the same point with twice the TV weight is not a minimiser of that objective
    P2 = so.Problem(g, pr["b"], lam=1.0, alpha=10.0, beta=10.0, tv=tv)
    f2 = so.objective(P2, xstar)
    assert min(so.objective(P2, xstar + 1e-3 * s * xstar) for s in (1, -1)) < f2


def _dense_circulant_apply(mu, x):
    return ci.circulant_apply(x, mu).ravel()


def test_mu_table_parts_against_dense_operators():
    """mu = gamma + alpha H_R + (beta^2/alpha) H_D + alpha kappa^2: each part is the
    spectrum of the matching circulant stand-in of a term of alpha A^T A, checked as an
    operator (so the frequency layout is checked too) against dense matrices."""
    Nm = 16
    g = op.Geometry(Nm, 24, 26)
    alpha, beta, kappa, gamma = 0.3, 1.7, 0.8, 0.25
    Lt = ci.Ltilde_matrix(Nm)
    lap = np.kron(np.eye(Nm), Lt) + np.kron(Lt, np.eye(Nm))
    x = np.random.default_rng(5).standard_normal((Nm, Nm))
    # D part: alpha (beta/alpha)^2 (I (x) L~ + L~ (x) I), the periodic D^T D of A's TV rows
    muD = ci.mu_table(g, alpha, beta, 0.0, c_r=0.0, h_dc=0.0)
    assert np.allclose(_dense_circulant_apply(muD, x), alpha * (beta / alpha) ** 2 * (lap @ x.ravel()), atol=1e-12)
    assert np.allclose(np.sort(muD.ravel()), np.sort(np.linalg.eigvalsh(alpha * (beta / alpha) ** 2 * lap)),
                       atol=1e-11)
    # gamma I and the nonnegativity row alpha kappa^2 I
    mu_g = ci.mu_table(g, alpha, 0.0, gamma, c_r=0.0, h_dc=0.0, kappa=kappa)
    assert np.allclose(_dense_circulant_apply(mu_g, x), (gamma + alpha * kappa * kappa) * x.ravel(), atol=1e-12)
    # projector part: alpha times the circulant with eigenvalues C_R / |nu| (eq. (circ_R)) and the DC entry;
    # on the constant image it is alpha h_dc, and h_dc is the Rayleigh quotient of K^T K there
    hdc = ci.h_dc_default(g)
    one = np.ones((Nm, Nm))
    assert hdc == pytest.approx(float(np.sum(op.K(one, g) ** 2)) / Nm ** 2, rel=1e-14)
    muR = ci.mu_table(g, alpha, 0.0, 0.0)
    assert np.allclose(ci.circulant_apply(one, muR), alpha * hdc * one, atol=1e-12)
    # a single Fourier mode (j, k) is scaled by alpha C_R / sqrt(j'^2 + k'^2)
    j, k = 3, 13
    jj, kk = np.meshgrid(np.arange(Nm), np.arange(Nm), indexing="ij")
    mode = np.cos(2 * math.pi * (j * jj + k * kk) / Nm)
    cr = ci.c_r_default(g)
    assert cr == pytest.approx(24 * Nm / math.pi, rel=1e-15)
    assert np.allclose(ci.circulant_apply(mode, muR), alpha * cr / math.hypot(3, 3) * mode, atol=1e-11)
    # and the whole table is the sum of its parts
    full = ci.mu_table(g, alpha, beta, gamma, kappa=kappa)
    parts = muD + mu_g + muR
    assert np.allclose(full, parts, rtol=1e-14)
