"""Pins of the oracle's solvers against the paper's exact reductions, lemmas
and optimality conditions:

* NCS with M = alpha A^T A reproduces the textbook (z, x, lambda) ADMM of the
  Appendix iterate for iterate (eq. (ADMM) vs eq. (NCS));
* the NCS fixed point is the dense-ADMM minimiser (Theorem 1);
* Lemma "monotone" and Lemma "summable" of Sec. 3.2 hold along the iterates;
* the power iterations match dense (generalised) eigenvalues, and after the
  rescale M >= alpha A^T A (assumption (A3));
* KKT conditions of the dual (eq. (dual)): A^T u* = 0, u* in dg(A x* - b).
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import circulant as ci
from oracle import operators as op
from oracle import solvers as so
import synth
from helpers import oproj

N, NA, ND = 16, 24, 26


@pytest.fixture(scope="module")
def ct16():
    pr = synth.ct_problem(0, N, NA, ND, 5, 0.01, oproj(N, NA, ND))
    return op.Geometry(N, NA, ND), pr["b"]


def dense_circulant(mu):
    n = mu.shape[0]
    F = np.exp(-2j * np.pi * np.outer(np.arange(n), np.arange(n)) / n)
    F2 = np.kron(F, F)
    return (np.linalg.inv(F2) @ np.diag(mu.ravel()) @ F2).real


@pytest.mark.parametrize("tv", ["aniso", "iso"])
def test_ncs_with_exact_inverse_is_textbook_admm(ct16, tv):
    g, b = ct16
    P = so.Problem(g, b, lam=0.5, alpha=0.7, beta=1.3, tv=tv)
    Ad = so.dense_A(P)
    xs_admm = so.admm_textbook(P, 30, Ad)
    st = so.zero_state(P)
    # Appendix: NCS's u^0 is the ADMM iterate prox_{alpha g*}(alpha (A x^0 - b - lambda^0)) at x^0 = lambda^0 = 0
    st.u = so.data_dual_prox(P, np.zeros_like(P.b), np.zeros_like(P.b))
    Minv = so.dense_Minv(P.alpha * Ad.T @ Ad)
    for k in range(30):
        st = so.ncs_step(P, st, Minv)
        assert np.linalg.norm(st.x - xs_admm[k]) <= 1e-11 * np.linalg.norm(xs_admm[k])


def test_power_iterations_match_dense_eigenvalues(ct16):
    g, b = ct16
    P = so.Problem(g, b, lam=0.5, alpha=1.0, beta=3.0)
    mu = ci.mu_table(g, P.alpha, P.beta, gamma=0.5)
    Ad = so.dense_A(P)
    AtA = Ad.T @ Ad
    Md = dense_circulant(mu)
    x0 = so.splitmix64_uniform(0, g.n).reshape(N, N)
    rho, _ = so.power_rho(P, mu, x0)
    ref = sla.eigh(P.alpha * AtA, Md, eigvals_only=True).max()
    assert rho == pytest.approx(ref, rel=1e-7)
    lm, _ = so.power_lmax_AtA(P, x0)
    assert lm == pytest.approx(np.linalg.eigvalsh(AtA).max(), rel=1e-7)
    # (A3) after the rescale, with margin
    mus, rho2 = so.a3_scaled_mu(P, mu)
    assert rho2 == pytest.approx(rho, rel=1e-12)
    assert np.linalg.eigvalsh(dense_circulant(mus) - P.alpha * AtA).min() >= 0.0
    # and PDHG's gamma satisfies gamma/alpha >= lambda_max(A^T A)
    gp, _ = so.pdhg_gamma(P)
    assert gp / P.alpha >= np.linalg.eigvalsh(AtA).max()


def test_splitmix64_reference_values():
    """First outputs of SplitMix64 seeded with 0 (the published generator:
    state += 0x9E3779B97F4A7C15 then two xor-shift-multiply rounds)."""
    golden = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    vals = so.splitmix64_uniform(0, 3)
    for v, g64 in zip(vals, golden):
        assert v == pytest.approx(2.0 * (g64 >> 11) / 2.0 ** 53 - 1.0, abs=0)


@pytest.fixture(scope="module")
def ct16_solution(ct16):
    g, b = ct16
    P = so.Problem(g, b, lam=0.5, alpha=1.0, beta=3.0, tv="aniso")
    mus, _ = so.a3_scaled_mu(P, ci.mu_table(g, 1.0, 3.0, 0.0))
    st = so.run(P, so.zero_state(P), 3500, so.circulant_Minv(mus))
    return P, mus, st


def test_ncs_fixed_point_is_admm_minimiser(ct16, ct16_solution):
    g, b = ct16
    P, mus, st = ct16_solution
    Pa = so.Problem(g, b, lam=0.5, alpha=10.0, beta=10.0, tv="aniso")
    xs = so.admm_textbook(Pa, 2500, so.dense_A(Pa))
    xstar = xs[-1]
    assert np.linalg.norm(st.x - xstar) <= 1e-8 * np.linalg.norm(xstar)
    assert so.objective(P, st.x) == pytest.approx(so.objective(Pa, xstar), rel=1e-12)


def test_kkt_at_ncs_limit(ct16_solution):
    P, mus, st = ct16_solution
    # u* = K x* - b (gradient of 1/2||.||^2), A^T u* = 0, |v*| <= lam alpha/beta
    assert np.linalg.norm(st.u - (op.K(st.x, P.g) - P.b)) <= 1e-8 * np.linalg.norm(st.u)
    r = so.AT_apply(P, st.u, st.vh, st.vv)
    assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(op.KT(st.u, P.g))
    rad = P.lam * P.alpha / P.beta
    assert np.abs(st.vh).max() <= rad * (1 + 1e-12) and np.abs(st.vv).max() <= rad * (1 + 1e-12)


def test_lemmas_monotone_and_summable(ct16_solution):
    """Sec. 3.2: D(x^{k+1}-x^k, u^{k+1}-u^k) and D(x^k - x*, u^k - u*) are
    nonincreasing, and D^2(step k) <= D^2(x^0 - x*, u^0 - u*)/(k+1)."""
    P, mus, sol = ct16_solution
    Mapply = lambda x: ci.circulant_apply(x, mus)
    st = so.zero_state(P)
    d0 = so.seminorm_sq(P, Mapply, st.x - sol.x, st.u - sol.u, st.vh - sol.vh, st.vv - sol.vv)
    prev_step = np.inf
    prev_dist = d0
    for k in range(200):
        nxt = so.ncs_step(P, st, so.circulant_Minv(mus))
        step = so.seminorm_sq(P, Mapply, nxt.x - st.x, nxt.u - st.u, nxt.vh - st.vh, nxt.vv - st.vv)
        dist = so.seminorm_sq(P, Mapply, nxt.x - sol.x, nxt.u - sol.u, nxt.vh - sol.vh, nxt.vv - sol.vv)
        assert step >= -1e-9 * d0                        # seminorm: nonnegative under (A3)
        assert step <= prev_step * (1 + 1e-9) + 1e-12 * d0
        assert dist <= prev_dist * (1 + 1e-9) + 1e-12 * d0
        assert step <= d0 / (k + 1) * (1 + 1e-9)
        prev_step, prev_dist, st = step, dist, nxt


def test_pdhg_converges_to_same_minimiser(ct16, ct16_solution):
    P, mus, sol = ct16_solution
    gp, _ = so.pdhg_gamma(P)
    st = so.zero_state(P)
    for _ in range(3000):
        st = so.pdhg_step(P, st, gp)
    assert np.linalg.norm(st.x - sol.x) <= 1e-4 * np.linalg.norm(sol.x)


def test_pet_kkt_at_ncs_limit():
    """TV-PET with the nonnegativity row (Sec. 4.2): at the limit the data dual is
    the likelihood gradient 1 - b/(K x + r), A^T u = 0, s <= 0, s x = 0, x >= 0."""
    pp = synth.pet_problem(0, 16, 24, 17, 5, oproj(16, 24, 17), total_counts=1e4)
    g = op.Geometry(16, 24, 17)
    P = so.Problem(g, pp["b"], lam=0.02, alpha=0.1, beta=0.1, kind="pet", kappa=1.0, r_bg=pp["r_bg"])
    mus, _ = so.a3_scaled_mu(P, ci.mu_table(g, 0.1, 0.1, 0.0, kappa=1.0))
    st = so.run(P, so.zero_state(P), 2500, so.circulant_Minv(mus))
    mu_y = op.K(st.x, g) + P.r_bg
    grad = 1.0 - P.b / mu_y
    assert np.linalg.norm(st.u - grad) <= 1e-6 * np.linalg.norm(grad)
    r = so.AT_apply(P, st.u, st.vh, st.vv, st.s)
    assert np.linalg.norm(r) <= 1e-6 * np.linalg.norm(op.KT(st.u, g))
    assert st.s.max() <= 0.0
    assert st.x.min() >= -1e-6 * st.x.max()
    assert np.abs(st.s * st.x).max() <= 1e-6 * np.abs(st.s).max() * st.x.max()
    # objective of the limit is no larger than at nearby feasible perturbations
    f = so.objective(P, st.x)
    rng = np.random.default_rng(0)
    for _ in range(5):
        assert so.objective(P, np.maximum(st.x + 1e-3 * rng.standard_normal(st.x.shape), 0)) >= f - 1e-9 * abs(f)


@pytest.mark.parametrize("tv", ["aniso", "iso"])
def test_admm_pcg_with_long_inner_loop_is_textbook_admm(ct16, tv):
    """The ADMM comparator with its PCG inner loop (circulant preconditioner) run to
    convergence inside every outer step reproduces the dense-pseudo-inverse ADMM of the
    Appendix; with a short inner loop it still descends to the same minimiser."""
    g, b = ct16
    P = so.Problem(g, b, lam=0.5, alpha=0.7, beta=1.3, tv=tv)
    Ad = so.dense_A(P)
    ref = so.admm_textbook(P, 8, Ad)
    mus, _ = so.a3_scaled_mu(P, ci.mu_table(g, P.alpha, P.beta, 0.0))
    xs = so.admm_pcg(P, 8, 120, so.circulant_Minv(mus))
    for k in range(8):
        assert np.linalg.norm(xs[k] - ref[k]) <= 1e-9 * np.linalg.norm(ref[k])


def test_admm_pcg_with_short_inner_loop_reaches_the_ncs_minimiser(ct16, ct16_solution):
    g, b = ct16
    P, mus, st = ct16_solution
    xs = so.admm_pcg(P, 1000, 3, so.circulant_Minv(mus))
    f_admm = so.objective(P, xs[-1])
    f_ncs = so.objective(P, st.x)
    assert 0.0 <= (f_admm - f_ncs) / f_ncs <= 1e-6
    assert np.linalg.norm(xs[-1] - st.x) <= 1e-5 * np.linalg.norm(st.x)
