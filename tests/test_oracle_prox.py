"""Pins of the oracle's proximal maps: Moreau's identity (eq. (Moreau))
against a direct argmin by bisection, the closed form S(u; c) of Sec. 4.2 as
the root of its quadratic, S(u; 0) = min(u, 1), and idempotence of the
projections."""
import numpy as np
import pytest

from oracle import prox


def argmin_1d(grad, lo, hi, iters=200):
    """Root of a monotone increasing derivative on [lo, hi] by bisection."""
    lo = np.array(lo, dtype=np.float64)
    hi = np.array(hi, dtype=np.float64)
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        g = grad(mid)
        lo = np.where(g < 0, mid, lo)
        hi = np.where(g < 0, hi, mid)
    return 0.5 * (lo + hi)


@pytest.mark.parametrize("alpha", [0.01, 0.3, 2.0])
def test_moreau_l2(alpha):
    z = np.random.default_rng(0).normal(0, 5, 200)
    # primal prox of (1/alpha) * 1/2 y^2 by bisection on its derivative
    w = z / alpha
    p = argmin_1d(lambda y: y / alpha + (y - w), -1e3, 1e3)
    assert np.allclose(prox.prox_l2_conj(z, alpha), z - alpha * p, atol=1e-9)


@pytest.mark.parametrize("alpha,t", [(0.5, 0.2), (0.01, 1.5)])
def test_moreau_l1_is_clip(alpha, t):
    """prox of alpha times the conjugate of t||.||_1 is the clip to [-t, t]."""
    z = np.random.default_rng(1).normal(0, 2, 300)
    p = prox.soft(z / alpha, t / alpha)
    assert np.allclose(prox.clip(z, t), z - alpha * p, atol=1e-12)


def test_moreau_iso_is_ball_projection():
    rng = np.random.default_rng(2)
    zh, zv = rng.normal(0, 1, (2, 50))
    alpha, t = 0.7, 0.4
    ph, pv = prox.soft_iso(zh / alpha, zv / alpha, t / alpha)
    bh, bv = prox.ball2(zh, zv, t)
    assert np.allclose(bh, zh - alpha * ph, atol=1e-12)
    assert np.allclose(bv, zv - alpha * pv, atol=1e-12)


@pytest.mark.parametrize("alpha", [1e-3, 0.1, 1.0])
def test_S_is_moreau_of_poisson_likelihood(alpha):
    """S(z; alpha b) = z - alpha prox_{(1/alpha) l}(z / alpha) with
    l(y; b) = y - b log y (b > 0) or y + indicator(y >= 0) (b = 0)."""
    rng = np.random.default_rng(3)
    z = rng.normal(0, 3, 400)
    b = rng.poisson(5.0, 400).astype(np.float64)
    w = z / alpha
    # derivative of (1/alpha) l(y) + 1/2 (y - w)^2 in y > 0
    grad = lambda y: (1.0 - b / y) / alpha + (y - w)
    y = argmin_1d(grad, np.full_like(z, 1e-300), np.full_like(z, 1e6))
    pos = b > 0
    ref = z - alpha * y
    # b = 0: the prox is max(w - 1/alpha, 0)
    ref0 = z - alpha * np.maximum(w - 1.0 / alpha, 0.0)
    ref = np.where(pos, ref, ref0)
    assert np.allclose(prox.S_kl(z, alpha * b), ref, rtol=1e-8, atol=1e-8)


def test_S_special_cases_and_quadratic():
    z = np.linspace(-5, 5, 101)
    assert np.allclose(prox.S_kl(z, 0.0), np.minimum(z, 1.0), atol=1e-15)
    c = 0.37
    w = prox.S_kl(z, c)
    assert np.all(w < 1.0)
    assert np.allclose((w - z) * (1.0 - w) + c, 0.0, atol=1e-12)


def test_projections_idempotent():
    rng = np.random.default_rng(4)
    z = rng.normal(0, 3, 100)
    assert np.array_equal(prox.clip(prox.clip(z, 1.2), 1.2), prox.clip(z, 1.2))
    assert np.array_equal(prox.min0(prox.min0(z)), prox.min0(z))
    h, v = prox.ball2(z[:50], z[50:], 0.8)
    h2, v2 = prox.ball2(h, v, 0.8)
    assert np.allclose(h, h2) and np.allclose(v, v2)
    assert np.all(np.sqrt(h * h + v * v) <= 0.8 + 1e-15)
