"""The 64x64 parallel-beam TV-CT workload (90 angles on [0, pi), 92 unit bins, 10 seeded
ellipses, 1% noise, lambda 0.01, anisotropic TV) in FP64, as the paper runs its small
comparisons (Sec. 5): NCS against PDHG (eq. (PDHG)) and against ADMM with an explicit
(A^T A)^+ (eq. (ADMM), the Appendix's textbook form).

* Theorem 1: the NCS fixed point is the minimiser, here the limit of the explicit-inverse
  ADMM, to 1e-8 relative.
* 500 iterations of each method at its best step on the paper's {1,3} x 10^p grid
  (NCS alpha 0.03, PDHG 0.01, ADMM 0.3; measured gaps 1.0e-6, 9.5e-4 and 5.5e-11): the
  explicit inverse is the per-iteration ideal that NCS approaches at PDHG's cost per
  iteration, and NCS is far ahead of PDHG.
"""
import numpy as np
import pytest

from oracle import circulant as ci
from oracle import operators as op
from oracle import solvers as so
import synth
from helpers import oproj

pytestmark = pytest.mark.slow


@pytest.fixture(scope="module")
def ct64():
    W = synth.WORKLOADS["ct64"]
    N, na, nd = W["N"], W["n_angles"], W["n_det"]
    assert (N, na, nd, W["lam"], W["tv"]) == (64, 90, 92, 0.01, "aniso")
    pr = synth.ct_problem(0, N, na, nd, W["n_ellipses"], W["noise_frac"], oproj(N, na, nd))
    g = op.Geometry(N, na, nd)
    mk = lambda a: so.Problem(g, pr["b"], lam=W["lam"], alpha=a, beta=a, tv=W["tv"])
    # A = [K; (beta/alpha) D] depends on beta/alpha only, here 1 for every method
    Ad = so.dense_A(mk(1.0))
    AtA = Ad.T @ Ad
    del Ad
    ev = np.linalg.eigvalsh(AtA)
    assert ev.min() > 0.0                        # K has full column rank: (A^T A)^+ is the inverse
    return mk, AtA, ev.max()


def test_config64_ncs_pdhg_and_explicit_admm(ct64):
    mk, AtA, lmax = ct64
    inv = so.explicit_inverse(AtA)
    assert np.allclose(inv @ AtA, np.eye(AtA.shape[0]), atol=1e-9)
    # explicit-inverse ADMM: 500 iterations, then on to its limit x*
    Pa = mk(0.3)
    at500 = {}
    xs = so.admm_explicit(Pa, 1500, inv, record=lambda k, x: at500.setdefault(k, x.copy()) if k == 499 else None)
    xstar = xs[-1]
    assert np.linalg.norm(xs[-1] - xs[-101]) <= 1e-12 * np.linalg.norm(xstar)
    fstar = so.objective(Pa, xstar)
    gap = lambda P, x: (so.objective(P, x) - fstar) / fstar
    g_admm = gap(Pa, at500[499])
    # NCS with the circulant M of eqs. (circ_R), (circ_D), rescaled for (A3)
    Pn = mk(0.03)
    mus, rho = so.a3_scaled_mu(Pn, ci.mu_table(Pn.g, 0.03, 0.03, 0.0))
    Minv = so.circulant_Minv(mus)
    st = so.run(Pn, so.zero_state(Pn), 500, Minv)
    g_ncs = gap(Pn, st.x)
    st = so.run(Pn, st, 3500, Minv)
    assert np.linalg.norm(st.x - xstar) <= 1e-8 * np.linalg.norm(xstar)
    # PDHG with gamma_P = alpha lambda_max(A^T A) (1 + 1e-2), lambda_max from the dense A^T A
    Pp = mk(0.01)
    gp = Pp.alpha * lmax * (1.0 + 1e-2)
    sp = so.zero_state(Pp)
    for _ in range(500):
        sp = so.pdhg_step(Pp, sp, gp)
    g_pdhg = gap(Pp, sp.x)
    assert 0.0 <= g_admm < g_ncs < 1e-5
    assert g_pdhg > 100.0 * g_ncs
