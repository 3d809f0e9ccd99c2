"""GPU ADMM comparator (admm_solve: the Appendix's textbook ADMM with A = [K; (beta/alpha) D]
and an x-update by conjugate gradients preconditioned by the circulant M, as in Sec. 1.3)
against the FP64 oracle's admm_pcg from the same zero state, through the C ABI.

Tolerances: one outer step composes the z prox, one A^T, n_cg + 1 products with A^T A and
n_cg + 1 circulant solves, each within 1e-5 of FP64 (the operator tests).  Conjugate
gradients is not a nonexpansive map, and its step lengths are ratios of dot products that
rounding perturbs to first order, so the bound is looser than the NCS iterations' 2e-5 per
step: 2e-4 after one outer step, 2e-3 after five.  A wrong sign, term or index gives
relative errors of order one.  The solve test runs to the 1e-4 gap against the oracle's f*
of the 64x64 workload and checks the returned image in FP64 with the oracle."""
import json
import os

import numpy as np
import pytest

import synth
from helpers import f32, oproj, oracle_scaled_mu, rel_l2, to_np
from oracle import operators as oop
from oracle import solvers as osv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("N,na,nd,tv", [(64, 90, 92, "aniso"), (48, 60, 70, "iso")])
def test_admm_iterates_match_oracle(N, na, nd, tv):
    import paper_1810_13100_gb300 as ncs
    lam, a, n_cg = 0.01, 0.1, 3
    pr = synth.ct_problem(0, N, na, nd, 8, 0.01, oproj(N, na, nd))
    P = osv.Problem(oop.Geometry(N, na, nd), f32(pr["b"]), lam=lam, alpha=a, beta=a, tv=tv)
    mus, _ = oracle_scaled_mu(N, na, nd, a, a, 0.0, tv)
    xs = osv.admm_pcg(P, 5, n_cg, osv.circulant_Minv(mus))
    plan = ncs.Plan(N, na, nd, lam, a, beta=a, tv=tv, power_tol=1e-9)
    b = torch.from_numpy(pr["b"].ravel()).cuda()
    x = torch.zeros(N * N, device="cuda")
    for k, tol in ((1, 2e-4), (5, 2e-3)):
        x.zero_()
        rep = plan.admm_solve(b, x, tol=0.0, max_outer=k, n_cg=n_cg)
        assert rep["iters"] == k
        err = rel_l2(to_np(x), xs[k - 1])
        assert err <= tol, (k, err)
    plan.close()


def test_admm_solve_reaches_gap_checked_by_oracle():
    import paper_1810_13100_gb300 as ncs
    W = synth.WORKLOADS["ct64"]
    N, na, nd = W["N"], W["n_angles"], W["n_det"]
    pr = synth.ct_problem(0, N, na, nd, W["n_ellipses"], W["noise_frac"], oproj(N, na, nd))
    with open(os.path.join(ROOT, "tests", "golden", "fstar_ct64_s0.json")) as fh:
        fs = json.load(fh)["f_star"]
    P = osv.Problem(oop.Geometry(N, na, nd), f32(pr["b"]), lam=W["lam"], alpha=0.1, beta=0.1, tv=W["tv"])
    plan = ncs.Plan(N, na, nd, W["lam"], 0.1, beta=0.1, tv=W["tv"])
    b = torch.from_numpy(pr["b"].ravel()).cuda()
    x = torch.zeros(N * N, device="cuda")
    rep = plan.admm_solve(b, x, tol=1e-4, max_outer=3000, n_cg=3, f_star=fs)
    assert rep["status"] == 0 and rep["gap"] <= 1e-4, rep
    f_oracle = osv.objective(P, x.double().cpu().numpy().reshape(N, N))
    assert fs * (1 - 1e-6) <= f_oracle <= fs * (1 + 1e-4 + 1e-6)
    assert rep["f"] == pytest.approx(f_oracle, rel=1e-6)
    plan.close()


def test_admm_rejects_unsupported_plans():
    import paper_1810_13100_gb300 as ncs
    N, na, nd = 32, 40, 46
    plan = ncs.Plan(N, na, nd, 0.01, 1.0, data="kl", nonneg=True)
    b = torch.ones(na * nd, device="cuda")
    x = torch.zeros(N * N, device="cuda")
    with pytest.raises(ncs.NCSError) as e:
        plan.admm_solve(b, x, max_outer=2)
    assert e.value.code == ncs.binding.NCS_ERR_UNSUPPORTED
    with pytest.raises(ncs.NCSError) as e:
        plan2 = ncs.Plan(N, na, nd, 0.01, 0.1)
        try:
            plan2.admm_solve(b, x, max_outer=2, n_cg=0)
        finally:
            plan2.close()
    assert e.value.code == ncs.binding.NCS_ERR_BADARG
    plan.close()
