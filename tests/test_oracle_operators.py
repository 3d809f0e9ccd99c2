"""Pins of the oracle's Joseph projector and finite differences against what
the mathematics fixes: adjointness, dense transposes, closed forms at
theta = 0 and pi/2, the analytic Radon transform of an ellipse (eq.
(radon-def)), and the Kronecker structure of D_2 (Sec. 2)."""
import math

import numpy as np
import pytest

from oracle import operators as op
from oracle import circulant as ci
import synth
from synth.phantom import Ellipses


GEOMS = [
    (64, 90, 92),      # 64x64 workload geometry
    (17, 13, 25),      # odd image side, odd angle count
    (32, 48, 47),      # odd bin count
    (20, 16, 30),      # angle count divisible by 4 (ties at pi/4, 3pi/4)
]


@pytest.mark.parametrize("N,na,nd", GEOMS)
def test_adjoint_fp64(N, na, nd):
    g = op.Geometry(N, na, nd)
    rng = np.random.default_rng(N * 1000 + na)
    for _ in range(3):
        x = rng.standard_normal((N, N))
        y = rng.standard_normal((na, nd))
        lhs = np.sum(op.K(x, g) * y)
        rhs = np.sum(x * op.KT(y, g))
        assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + np.linalg.norm(x) * np.linalg.norm(y))


def test_adjoint_user_angles_and_offset():
    th = np.array([0.0, 0.3, math.pi / 4, 1.1, math.pi / 2, 2.0, 3 * math.pi / 4, 3.0])
    g = op.Geometry(24, len(th), 37, spacing=1.3, offset=0.4, theta=th)
    rng = np.random.default_rng(5)
    x = rng.standard_normal((24, 24))
    y = rng.standard_normal((len(th), 37))
    lhs, rhs = np.sum(op.K(x, g) * y), np.sum(x * op.KT(y, g))
    assert abs(lhs - rhs) <= 1e-13 * np.linalg.norm(x) * np.linalg.norm(y)


def test_dense_transpose_16():
    g = op.Geometry(16, 8, 23)
    Kd = op.dense_of(lambda e: op.K(e.reshape(16, 16), g), 256)
    KTd = op.dense_of(lambda e: op.KT(e.reshape(8, 23), g), 8 * 23)
    assert np.max(np.abs(KTd - Kd.T)) <= 1e-14 * np.max(np.abs(Kd))
    # at most two nonzeros per (ray, step): row sums of |K| bounded by the chord cover
    assert np.all(np.count_nonzero(Kd, axis=1) <= 2 * 16)


@pytest.mark.parametrize("N,nd", [(64, 92), (512, 730), (16, 20)])
def test_theta0_is_column_sums(N, nd):
    """theta = 0: rays are the lines u = s_t; with N and n_det both even the bins
    sit on pixel columns, so K x at a = 0 is exactly a column sum."""
    g = op.Geometry(N, 4, nd)
    x = np.random.default_rng(0).standard_normal((N, N))
    y0 = op.K(x, g)[0]
    off = (nd - N) // 2
    assert np.max(np.abs(y0[off:off + N] - x.sum(axis=0))) <= 1e-12 * N
    assert np.all(y0[:off] == 0) and np.all(y0[off + N:] == 0)


def test_theta0_odd_bins_is_mean_of_adjacent_columns():
    N, nd = 256, 257
    g = op.Geometry(N, 180, nd)
    x = np.random.default_rng(1).standard_normal((N, N))
    y0 = op.K(x, g)[0]
    cs = np.concatenate([[0.0], x.sum(axis=0), [0.0]])
    expect = 0.5 * (cs[:-1] + cs[1:])
    assert np.max(np.abs(y0 - expect)) <= 1e-11


def test_theta_half_pi_is_row_sums():
    """theta = pi/2: rays are v = s_t, stepped over columns, bin t on row
    j = (N + n_det)/2 - 1 - t."""
    N, na, nd = 64, 90, 92
    g = op.Geometry(N, na, nd)
    x = np.random.default_rng(2).standard_normal((N, N))
    y = op.K(x, g)[na // 2]
    t = np.arange(nd)
    j = (N + nd) // 2 - 1 - t
    ok = (j >= 0) & (j < N)
    assert np.max(np.abs(y[ok] - x.sum(axis=1)[j[ok]])) <= 1e-12 * N
    assert np.all(y[~ok] == 0)


def test_branch_rule_ties_go_to_rows():
    g = op.Geometry(8, 20, 10)
    a = np.arange(20)
    assert g.row_branch[5] == 1 and g.row_branch[15] == 1       # pi/4, 3pi/4
    assert np.all(g.row_branch[(a > 5) & (a < 15)] == 0)
    assert np.all(g.row_branch[(a <= 5) | (a >= 15)] == 1)


def test_ellipse_chord_formula_brute_force():
    """The generator's closed-form chord length agrees with brute-force sampling
    along the line (so the analytic sinogram is an independent reference)."""
    ell = Ellipses(np.array([0.25]), np.array([-0.1]), np.array([0.45]), np.array([0.2]),
                   np.array([0.7]), np.array([0.8]))
    N = 100
    for th in (0.1, 1.0, 2.2):
        for s_pix in (-20.0, 3.0, 15.5):
            val = synth.radon_ellipses(ell, N, np.array([th]), np.array([s_pix]))[0, 0]
            s = s_pix * 2.0 / N
            tt = np.linspace(-2, 2, 400001)
            px = s * math.cos(th) - tt * math.sin(th)
            py = s * math.sin(th) + tt * math.cos(th)
            du, dv = px - 0.25, py + 0.1
            c, sn = math.cos(0.7), math.sin(0.7)
            p = (du * c + dv * sn) / 0.45
            q = (-du * sn + dv * c) / 0.2
            inside = (p * p + q * q <= 1.0).sum() * (tt[1] - tt[0])
            assert abs(val - 0.8 * inside * N / 2) <= 1e-3 * N


def test_projector_converges_to_analytic_radon():
    """K of the rasterised ellipse approaches the exact line integrals of eq.
    (radon-def) as the grid refines; the mirrored orientation does not."""
    ell = Ellipses(np.array([0.3]), np.array([-0.2]), np.array([0.4]), np.array([0.15]),
                   np.array([0.6]), np.array([1.0]))
    errs = []
    for N in (32, 64, 128):
        na, nd = 36, (3 * N // 4) * 2
        g = op.Geometry(N, na, nd)
        Kx = op.K(synth.rasterize(ell, N), g)
        R = synth.radon_ellipses(ell, N, synth.angles(na), synth.det_centres(nd))
        errs.append(np.linalg.norm(Kx - R) / np.linalg.norm(R))
        mirror = Ellipses(ell.cx, -ell.cy, ell.ax, ell.ay, -ell.phi, ell.rho)
        Rm = synth.radon_ellipses(mirror, N, synth.angles(na), synth.det_centres(nd))
        assert np.linalg.norm(Kx - Rm) / np.linalg.norm(R) > 0.5
    assert errs[2] < 0.03
    assert errs[1] < 0.65 * errs[0] and errs[2] < 0.65 * errs[1]


def test_D_dense_and_kron():
    N = 8
    x = np.random.default_rng(3).standard_normal((N, N))
    dh, dv = op.D(x)
    Dn = op.D1_matrix(N)
    D2 = np.vstack([np.kron(np.eye(N), Dn), np.kron(Dn, np.eye(N))])
    assert np.allclose(np.concatenate([dh.ravel(), dv.ravel()]), D2 @ x.ravel(), atol=1e-14)
    DTd = op.dense_of(lambda w: op.DT(w[:N * (N - 1)].reshape(N, N - 1), w[N * (N - 1):].reshape(N - 1, N)),
                      2 * N * (N - 1))
    assert np.max(np.abs(DTd - D2.T)) == 0.0
    # D^T D 1 = 0 and L_n = D_n^T D_n has the printed tridiagonal form (Sec. 2)
    assert np.max(np.abs(op.DT(*op.D(np.ones((N, N)))))) == 0.0
    Ln = Dn.T @ Dn
    assert Ln[0, 0] == 1 and Ln[-1, -1] == 1 and np.all(np.diag(Ln)[1:-1] == 2)
    assert np.all(np.diag(Ln, 1) == -1)


def test_D2TD2_dominated_by_periodic_laplacian():
    """D_2^T D_2 <= I (x) L~ + L~ (x) I, since L~_n - L_n = (e1 - en)(e1 - en)^T >= 0."""
    N = 10
    Dn = op.D1_matrix(N)
    D2 = np.vstack([np.kron(np.eye(N), Dn), np.kron(Dn, np.eye(N))])
    Lt = ci.Ltilde_matrix(N)
    P = np.kron(np.eye(N), Lt) + np.kron(Lt, np.eye(N))
    assert np.linalg.eigvalsh(P - D2.T @ D2).min() >= -1e-12


def test_ramlak_zero_dc_gain_and_fbp_reconstructs_a_disk():
    """The Ram-Lak kernel sums to zero (its transfer function vanishes at DC:
    1/4 - (2/pi^2) sum_{odd n} 1/n^2 = 0), and FBP of the exact sinogram of a disk
    returns the disk (inside ~1, outside ~0)."""
    from oracle import fbp
    h = fbp.ramlak(200001)
    assert abs(h.sum()) < 1e-5
    N, na, nd = 128, 180, 184
    disk = Ellipses(np.array([0.1]), np.array([-0.05]), np.array([0.5]), np.array([0.5]),
                    np.array([0.0]), np.array([1.0]))
    g = op.Geometry(N, na, nd)
    sino = synth.radon_ellipses(disk, N, synth.angles(na), synth.det_centres(nd))
    rec = fbp.fbp(sino, g)
    truth = synth.rasterize(disk, N)
    from scipy.ndimage import binary_erosion
    inside = binary_erosion(truth > 0.5, iterations=3)
    outside = binary_erosion(truth < 0.5, iterations=3)
    assert abs(rec[inside].mean() - 1.0) < 0.03
    assert abs(rec[outside].mean()) < 0.03
