"""Pins of the oracle's fan-beam projector (Sec. 4, fan beam geometry) to facts that do
not come from its own formulas:

- far-source limit: with the source at distance R -> infinity and the fan pitch d/R, every
  view is a parallel-beam projection with bin pitch d, so the fan projector must agree
  with the (separately pinned) parallel-beam Joseph projector;
- rotation: turning the object by 90 degrees turns its sinogram by a quarter of the views
  (the pixel grid maps onto itself), which fixes the view and ray orientation;
- a single bright pixel lands, in every view, on the channel whose fan angle is the angle
  between the central ray and the line from the source to that pixel (computed here from
  the source position, independently of the ray parameters);
- the projection of an all-ones image is the length of the ray's chord through the image
  square, up to Joseph's partial first and last steps (at most two steps of length
  <= sqrt(2));
- K^T is the transpose of K."""
import math

import numpy as np
import pytest

from oracle import operators as oop


def cover_pitch(N, R, nd, slack=1.05):
    """Fan pitch whose fan just covers the image's circumscribed circle (with slack)."""
    return 2.0 * math.asin(N / math.sqrt(2.0) / R) / nd * slack


def test_far_source_limit_is_parallel_beam():
    N, na, nd, d = 32, 30, 48, 1.0
    R = 1e9
    beta = np.arange(na) * (math.pi / na)
    fan = oop.FanGeometry(N, na, nd, R, d / R, beta=beta)
    par = oop.Geometry(N, na, nd)
    x = np.random.default_rng(0).random((N, N))
    yf, yp = oop.K(x, fan), oop.K(x, par)
    assert np.linalg.norm(yf - yp) / np.linalg.norm(yp) < 1e-6
    assert np.array_equal(fan.row_branch.reshape(na, nd)[:, 0], par.row_branch)


def test_quarter_turn_of_object_shifts_views():
    N, na, nd, R = 24, 36, 40, 40.0
    g = oop.FanGeometry(N, na, nd, R, cover_pitch(N, R, nd))
    x = np.random.default_rng(1).random((N, N))
    y = oop.K(x, g)
    y_rot = oop.K(np.rot90(x), g)           # object turned counter-clockwise by 90 degrees
    q = na // 4
    assert np.max(np.abs(y_rot[q:] - y[:-q])) < 1e-12 * np.max(np.abs(y))
    assert np.max(np.abs(y_rot[:q] - y[-q:])) < 1e-12 * np.max(np.abs(y))


def test_point_object_lands_on_its_channel():
    N, na, nd, R = 64, 16, 128, 100.0
    pitch = cover_pitch(N, R, nd)
    g = oop.FanGeometry(N, na, nd, R, pitch, offset=0.3 * pitch)
    j, i = 12, 49                            # well off the centre: a mirrored fan angle would miss
    x = np.zeros((N, N))
    x[j, i] = 1.0
    y = oop.K(x, g)
    cN = 0.5 * (N - 1)
    P = (i - cN, cN - j)
    for a in range(na):
        Su, Sv = g.source(a)
        d0 = (-Su / R, -Sv / R)             # central ray direction
        du, dv = P[0] - Su, P[1] - Sv
        gam = math.atan2(d0[0] * dv - d0[1] * du, d0[0] * du + d0[1] * dv)
        t_star = (gam - g.offset) / pitch + 0.5 * (nd - 1)
        w = y[a]
        assert w.sum() > 0
        centroid = float(np.sum(np.arange(nd) * w) / np.sum(w))
        assert abs(centroid - t_star) < 0.3, (a, centroid, t_star)


def test_constant_image_gives_chord_lengths():
    N, na, nd, R = 48, 12, 80, 70.0
    g = oop.FanGeometry(N, na, nd, R, cover_pitch(N, R, nd))
    y = oop.K(np.ones((N, N)), g).ravel()
    h = N / 2.0                              # the image square [-h, h]^2 (pixel edges)
    for r in range(g.m):
        c, s, st = g.cos_r[r], g.sin_r[r], g.s_r[r]
        # chord of the line u c + v s = st through the square: parametrise p = st n + l e
        n, e = (c, s), (-s, c)
        lo, hi = -np.inf, np.inf
        for k in range(2):
            p0, dk = st * n[k], e[k]
            if abs(dk) < 1e-15:
                if abs(p0) > h:
                    lo, hi = 0.0, 0.0
                continue
            a1, a2 = (-h - p0) / dk, (h - p0) / dk
            lo, hi = max(lo, min(a1, a2)), min(hi, max(a1, a2))
        chord = max(0.0, hi - lo)
        assert abs(y[r] - chord) <= 2.0 * math.sqrt(2.0) + 1e-9, (r, y[r], chord)


def test_transpose_is_adjoint():
    N, na, nd, R = 40, 20, 64, 60.0
    g = oop.FanGeometry(N, na, nd, R, cover_pitch(N, R, nd))
    rng = np.random.default_rng(3)
    x, y = rng.random((N, N)), rng.random((na, nd))
    lhs, rhs = np.sum(oop.K(x, g) * y), np.sum(x * oop.KT(y, g))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_fan_ncs_fixed_point_is_dense_admm_minimiser():
    """NCS (eq. (NCS)) with the fan-beam K and M from eq. (H-fan) (least-squares form over
    probe images, rescaled for (A3)) converges to the minimiser that the textbook ADMM of the
    Appendix reaches with a dense (A^T A)^+; at the limit u* = K x* - b and A^T u* = 0."""
    from oracle import circulant as ci
    from oracle import solvers as so
    import synth
    N, na, nd, R = 16, 24, 28, 20.0
    g = oop.FanGeometry(N, na, nd, R, cover_pitch(N, R, nd))
    b = synth.ct_problem(0, N, na, nd, 4, 0.01, lambda x: oop.K(x, g))["b"].astype(np.float64)
    P = so.Problem(g, b, lam=0.5, alpha=1.0, beta=3.0, tv="aniso")
    vs = [so.splitmix64_uniform(1 + q, N * N).reshape(N, N) for q in range(8)]
    h = np.maximum(ci.probe_ls(lambda v: oop.KT(oop.K(v, g), g), N, vs), 0.0)
    h[0, 0] = ci.h_dc_default(g)
    mus, rho = so.a3_scaled_mu(P, P.alpha * h + (P.beta ** 2 / P.alpha) * ci.H_D(N))
    st = so.run(P, so.zero_state(P), 4000, so.circulant_Minv(mus))
    Pa = so.Problem(g, b, lam=0.5, alpha=10.0, beta=10.0, tv="aniso")
    xstar = so.admm_textbook(Pa, 2500, so.dense_A(Pa))[-1]
    assert np.linalg.norm(st.x - xstar) <= 1e-8 * np.linalg.norm(xstar)
    assert np.linalg.norm(st.u - (oop.K(st.x, g) - b)) <= 1e-8 * np.linalg.norm(st.u)
    r = so.AT_apply(P, st.u, st.vh, st.vv)
    assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(oop.KT(st.u, g))
