"""Pins of the oracle's 3-D cone-beam NCS (oracle/cone.py; Sec. 4, cone beam geometry) to facts
that do not come from its own formulas:

- a volume that is constant along z, seen by rays that stay inside its slices, projects like
  its 2-D image under the (separately pinned) fan-beam projector, times the path-length factor
  sqrt(1 + sigma^2) of the ray's slope;
- a single bright voxel lands, in every view, on the channel of its fan angle and on the row
  of its slope w / |P - S| seen from the source (both computed here from the source position);
- a constant volume projects to the length of each ray's chord through the volume's box, up to
  Joseph's partial first and last steps;
- K^T is the transpose of K, D^T of D, and D^T D annihilates constants;
- the 3-D H_D is the spectrum of the dense periodic 3-D Laplacian; the 3-D probe estimator
  recovers an exactly circulant operator;
- NCS converges to the minimiser that the textbook ADMM (Appendix) reaches with a dense
  (A^T A)^+, and satisfies the KKT conditions there."""
import math

import numpy as np
import pytest

from oracle import cone as oc
from oracle import operators as oop
from oracle import solvers as osv


def cover_pitch(N, R, nd, slack=1.05):
    return 2.0 * math.asin(N / math.sqrt(2.0) / R) / nd * slack


def test_z_constant_volume_projects_like_the_fan_beam():
    N, Nz, na, nr, nd, R = 24, 16, 12, 5, 40, 40.0
    g = oc.ConeGeometry(N, Nz, na, nr, nd, R, cover_pitch(N, R, nd), row_pitch=0.03)
    x2 = np.random.default_rng(0).random((N, N))
    y = oc.K(np.broadcast_to(x2, (Nz, N, N)), g)
    yf = oop.K(x2, g.fan)
    ref = np.sqrt(1.0 + g.sigma ** 2)[None, :, None] * yf[:, None, :]
    assert np.max(np.abs(y - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_transpose_is_adjoint():
    N, Nz, na, nr, nd, R = 20, 9, 10, 6, 36, 40.0
    g = oc.ConeGeometry(N, Nz, na, nr, nd, R, cover_pitch(N, R, nd), row_pitch=0.08, row_offset=0.01)
    rng = np.random.default_rng(1)
    x, y = rng.random(g.shape), rng.random(g.sino_shape)
    lhs, rhs = np.sum(oc.K(x, g) * y), np.sum(x * oc.KT(y, g))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_point_voxel_lands_on_its_channel_and_row():
    N, Nz, na, nr, nd, R = 48, 24, 16, 64, 96, 80.0
    pitch, row_pitch = cover_pitch(N, R, nd), 0.006
    g = oc.ConeGeometry(N, Nz, na, nr, nd, R, pitch, row_pitch, offset=0.2 * pitch, row_offset=0.3 * row_pitch)
    k, j, i = 17, 9, 33                      # off-centre in all three axes
    x = np.zeros(g.shape)
    x[k, j, i] = 1.0
    y = oc.K(x, g)
    cN, cZ = 0.5 * (N - 1), 0.5 * (Nz - 1)
    P = (i - cN, cN - j)
    w = k - cZ
    for a in range(na):
        Su, Sv = g.fan.source(a)
        d0 = (-Su / R, -Sv / R)
        du, dv = P[0] - Su, P[1] - Sv
        gam = math.atan2(d0[0] * dv - d0[1] * du, d0[0] * du + d0[1] * dv)
        t_star = (gam - g.offset) / pitch + 0.5 * (nd - 1)
        r_star = (w / math.hypot(du, dv) - g.row_offset) / row_pitch + 0.5 * (nr - 1)
        ya = y[a]
        assert ya.sum() > 0
        t_c = float(np.sum(np.arange(nd) * ya.sum(axis=0)) / ya.sum())
        r_c = float(np.sum(np.arange(nr) * ya.sum(axis=1)) / ya.sum())
        assert abs(t_c - t_star) < 0.3, (a, t_c, t_star)
        assert abs(r_c - r_star) < 0.3, (a, r_c, r_star)


def test_constant_volume_gives_chord_lengths():
    N, Nz, na, nr, nd, R = 32, 8, 6, 7, 48, 50.0
    g = oc.ConeGeometry(N, Nz, na, nr, nd, R, cover_pitch(N, R, nd), row_pitch=0.05)
    y = oc.K(np.ones(g.shape), g).ravel()
    h, hz = N / 2.0, Nz / 2.0
    for r in range(g.m):
        c, s, st, sg = g.cos_r[r], g.sin_r[r], g.s_r[r], g.sig_r[r]
        S = np.array([g.su_r[r], g.sv_r[r], 0.0])
        d = np.array([s, -c, sg]) / math.sqrt(1.0 + sg * sg)      # unit 3-D direction
        lo, hi = 0.0, np.inf
        for ax, half in ((0, h), (1, h), (2, hz)):
            if abs(d[ax]) < 1e-15:
                if abs(S[ax]) > half:
                    lo, hi = 0.0, 0.0
                continue
            a1, a2 = (-half - S[ax]) / d[ax], (half - S[ax]) / d[ax]
            lo, hi = max(lo, min(a1, a2)), min(hi, max(a1, a2))
        chord = max(0.0, hi - lo)
        step = math.sqrt(2.0) * math.sqrt(1.0 + sg * sg)
        assert abs(y[r] - chord) <= 2.0 * step + 1e-9, (r, y[r], chord)


def test_D_transpose_and_constants():
    rng = np.random.default_rng(2)
    Nz, N = 3, 4
    n = Nz * N * N
    Dd = np.stack([np.concatenate([c.ravel() for c in oc.D(e.reshape(Nz, N, N))]) for e in np.eye(n)], axis=1)
    m = Dd.shape[0]
    DTd = np.stack([oc.DT(*_split(e, Nz, N)).ravel() for e in np.eye(m)], axis=1)
    assert np.max(np.abs(DTd - Dd.T)) == 0.0
    assert np.max(np.abs(oc.DT(*oc.D(np.ones((Nz, N, N)))))) == 0.0
    x = rng.random((Nz, N, N))
    assert np.allclose(Dd @ x.ravel(), np.concatenate([c.ravel() for c in oc.D(x)]))


def _split(v, Nz, N):
    a, b = Nz * N * (N - 1), Nz * (N - 1) * N
    return (v[:a].reshape(Nz, N, N - 1), v[a:a + b].reshape(Nz, N - 1, N), v[a + b:].reshape(Nz - 1, N, N))


def test_H_D_is_the_periodic_3d_laplacian_spectrum():
    from oracle import circulant as oci
    N, Nz = 4, 3
    L = lambda n: oci.Ltilde_matrix(n)
    I = np.eye
    lap = np.kron(np.kron(L(Nz), I(N)), I(N)) + np.kron(np.kron(I(Nz), L(N)), I(N)) + np.kron(np.kron(I(Nz), I(N)), L(N))
    assert np.allclose(np.sort(np.linalg.eigvalsh(lap)), np.sort(oc.H_D(N, Nz).ravel()), atol=1e-12)


def test_probe_ls_recovers_a_circulant():
    shape = (3, 4, 4)
    h = np.random.default_rng(3).random(shape) + 0.5
    h = 0.5 * (h + np.roll(np.flip(h), 1, axis=(0, 1, 2)))     # even: a real operator
    vs = [osv.splitmix64_uniform(1 + q, h.size).reshape(shape) for q in range(3)]
    est = oc.probe_ls(lambda v: oc.circulant_apply(v, h), shape, vs)
    assert np.max(np.abs(est - h)) <= 1e-12 * h.max()


def test_cone_ncs_fixed_point_is_dense_admm_minimiser():
    import synth
    N, Nz, na, nr, nd, R = 8, 4, 12, 4, 12, 14.0
    g = oc.ConeGeometry(N, Nz, na, nr, nd, R, cover_pitch(N, R, nd), row_pitch=0.1)
    rng = np.random.default_rng(4)
    x_true = np.broadcast_to(synth.ct_phantom(0, N, 4, 4, 3)[0], (Nz, N, N)) * (1.0 + 0.1 * rng.random((Nz, 1, 1)))
    b = oc.K(x_true, g) + 0.01 * rng.standard_normal(g.sino_shape)
    P = oc.Problem(g, b, lam=0.5, alpha=1.0, beta=3.0, tv="aniso")
    mus, rho = oc.a3_scaled_mu(P, oc.mu_probes(P, 8))
    st = oc.run(P, oc.zero_state(P), 4000, lambda r: oc.circulant_solve(r, mus))
    Pa = oc.Problem(g, b, lam=0.5, alpha=10.0, beta=10.0, tv="aniso")
    xstar = oc.admm_textbook(Pa, 2500, oc.dense_A(Pa))
    assert np.linalg.norm(st.x - xstar) <= 1e-8 * np.linalg.norm(xstar)
    assert oc.objective(P, st.x) == pytest.approx(oc.objective(Pa, xstar), rel=1e-12)
    assert np.linalg.norm(st.u - (oc.K(st.x, g) - b)) <= 1e-8 * np.linalg.norm(st.u)
    r = oc.AT_apply(P, st.u, st.v)
    assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(oc.KT(st.u, g))


def test_ellipsoid_phantom_volume():
    """The 3-D phantom generator: a sphere of radius 1/2 at the centre fills (4/3) pi (1/2)^3
    of the [-1, 1]^3 volume's 8, and a rotation about w leaves a sphere unchanged."""
    import synth
    ell = synth.phantom.Ellipsoids(np.zeros((1, 3)), np.full((1, 3), 0.5), np.array([0.7]), np.array([2.0]))
    vol = synth.rasterize3(ell, 64, 64)
    frac = float(np.mean(vol > 0))
    assert abs(frac - (4.0 / 3.0) * math.pi * 0.125 / 8.0) < 0.02 * frac
    assert set(np.unique(vol)) <= {0.0, 2.0}
    ell0 = synth.phantom.Ellipsoids(np.zeros((1, 3)), np.full((1, 3), 0.5), np.array([0.0]), np.array([2.0]))
    assert np.array_equal(vol, synth.rasterize3(ell0, 64, 64))


def test_cone_pdhg_reaches_the_same_minimiser():
    """PDHG (eq. (PDHG), M = gamma_P I) on the same 3-D problem converges to the dense-ADMM
    minimiser too (slower: to 1e-4 after 4000 iterations)."""
    import synth
    N, Nz, na, nr, nd, R = 8, 4, 12, 4, 12, 14.0
    g = oc.ConeGeometry(N, Nz, na, nr, nd, R, cover_pitch(N, R, nd), row_pitch=0.1)
    rng = np.random.default_rng(4)
    x_true = np.broadcast_to(synth.ct_phantom(0, N, 4, 4, 3)[0], (Nz, N, N)) * (1.0 + 0.1 * rng.random((Nz, 1, 1)))
    b = oc.K(x_true, g) + 0.01 * rng.standard_normal(g.sino_shape)
    P = oc.Problem(g, b, lam=0.5, alpha=1.0, beta=3.0, tv="aniso")
    gp = oc.pdhg_gamma(P)
    st = oc.zero_state(P)
    for _ in range(4000):
        st = oc.pdhg_step(P, st, gp)
    Pa = oc.Problem(g, b, lam=0.5, alpha=10.0, beta=10.0, tv="aniso")
    xstar = oc.admm_textbook(Pa, 2500, oc.dense_A(Pa))
    assert np.linalg.norm(st.x - xstar) <= 1e-4 * np.linalg.norm(xstar)
    # gamma_P from the largest eigenvalue of the dense A^T A, times alpha (1 + 1e-2); the power
    # iteration's Rayleigh quotient approaches it from below
    lm_dense = float(np.linalg.eigvalsh(oc.dense_A(P).T @ oc.dense_A(P)).max())
    exact = P.alpha * lm_dense * 1.01
    assert exact * (1 - 1e-6) <= gp <= exact * (1 + 1e-12)
