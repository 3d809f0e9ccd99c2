"""GPU parity of whole NCS and PDHG iterations (all steps of one iteration:
gather A^T, FFT solve with M, primal update, forward projection with the data
prox, TV dual prox, nonnegativity prox) against the FP64 oracle from the same
zero state, through the C ABI.

Tolerances: one iteration composes the per-operator errors (<= 1e-5 each);
later iterates also carry the rounding of earlier ones through a nonexpansive
map (Sec. 3.2), so the bound grows at most linearly: 2e-5 after 1 iteration,
2e-4 after 20.  The TV dual v is a projection of v + beta D xbar, which is
nonexpansive but not relatively well conditioned (where D xbar is small its
direction is not), so its error is measured against the size of that argument,
||v|| + beta ||D xbar||, which bounds it."""
import numpy as np
import pytest

import synth
from helpers import f32, oproj, oracle_scaled_mu, rel_l2, to_np, v_to_oracle
from oracle import circulant as oci
from oracle import operators as oop
from oracle import solvers as osv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def run_pair(kind, N, na, nd, tv, lam, alpha, beta, iters, solver="ncs", seed=0, gamma=0.0):
    import paper_1810_13100_gb300 as ncs
    g = oop.Geometry(N, na, nd)
    if kind == "pet":
        pr = synth.pet_problem(seed, N, na, nd, 8, oproj(N, na, nd), total_counts=2e5)
        P = osv.Problem(g, f32(pr["b"]), lam=lam, alpha=alpha, beta=beta, kind="pet", tv=tv, kappa=1.0,
                        r_bg=f32(pr["r_bg"]))
        plan = ncs.Plan(N, na, nd, lam, alpha, beta=beta, tv=tv, data="kl", nonneg=True, gamma=gamma,
                        power_tol=1e-9)
        bg = torch.from_numpy(pr["r_bg"].ravel()).cuda()
    else:
        pr = synth.ct_problem(seed, N, na, nd, 8, 0.01, oproj(N, na, nd))
        P = osv.Problem(g, f32(pr["b"]), lam=lam, alpha=alpha, beta=beta, tv=tv)
        plan = ncs.Plan(N, na, nd, lam, alpha, beta=beta, tv=tv, gamma=gamma, power_tol=1e-9)
        bg = None
    b = torch.from_numpy(pr["b"].ravel()).cuda()
    x = torch.zeros(N * N, device="cuda")
    u = torch.zeros(na * nd, device="cuda")
    v = torch.zeros(2 * N * N, device="cuda")
    s = torch.zeros(N * N, device="cuda") if kind == "pet" else None
    st = osv.zero_state(P)
    if solver == "ncs":
        mus, _ = oracle_scaled_mu(N, na, nd, alpha, beta, gamma, tv, kappa=1.0 if kind == "pet" else 0.0,
                                  kind=kind)
        Minv = osv.circulant_Minv(mus)
        step = lambda s_: osv.ncs_step(P, s_, Minv)
        gpu_step = plan.step
    else:
        gp, _ = osv.pdhg_gamma(P)
        step = lambda s_: osv.pdhg_step(P, s_, gp)
        gpu_step = plan.pdhg_step
    out = []
    done = 0
    for k in iters:
        gpu_step(x, u, v, s, b, bg, n_iter=k - done)
        prev = st
        for _ in range(k - done):
            prev = st
            st = step(st)
        done = k
        torch.cuda.synchronize()
        vh, vv = v_to_oracle(to_np(v), N)
        dh, dv = oop.D(2.0 * st.x - prev.x)
        vref = np.concatenate([st.vh.ravel(), st.vv.ravel()])
        vscale = np.linalg.norm(vref) + beta * np.sqrt(np.sum(dh * dh) + np.sum(dv * dv))
        errs = dict(x=rel_l2(to_np(x), st.x), u=rel_l2(to_np(u), st.u),
                    v=np.linalg.norm(np.concatenate([vh.ravel(), vv.ravel()]) - vref) / max(vscale, 1e-300))
        if s is not None:
            sscale = np.linalg.norm(st.s) + alpha * np.linalg.norm(2.0 * st.x - prev.x)
            errs["s"] = np.linalg.norm(to_np(s) - st.s.ravel()) / max(sscale, 1e-300)
        out.append((k, errs))
    plan.close()
    return out


@pytest.mark.parametrize("N,na,nd,tv", [(48, 60, 70, "aniso"), (96, 140, 130, "iso"), (64, 90, 92, "aniso")])
def test_ncs_iterations_ct(N, na, nd, tv):
    for k, errs in run_pair("ct", N, na, nd, tv, lam=0.3, alpha=1.0, beta=3.0, iters=[1, 5, 20]):
        tol = 2e-5 if k == 1 else 2e-4
        for name, e in errs.items():
            assert e <= tol, (k, name, e)


def test_ncs_iterations_ct_with_gamma_and_radix3():
    for k, errs in run_pair("ct", 96, 100, 98, "iso", lam=0.3, alpha=0.5, beta=1.0, iters=[1, 10], gamma=2.0):
        for name, e in errs.items():
            assert e <= (2e-5 if k == 1 else 2e-4), (k, name, e)


def test_ncs_iterations_pet():
    for k, errs in run_pair("pet", 48, 60, 70, "aniso", lam=0.02, alpha=0.1, beta=0.1, iters=[1, 5, 20]):
        for name, e in errs.items():
            assert e <= (2e-5 if k == 1 else 2e-4), (k, name, e)


@pytest.mark.parametrize("kind,tv", [("ct", "iso"), ("pet", "aniso")])
def test_pdhg_iterations(kind, tv):
    lam, alpha, beta = (0.3, 1.0, 3.0) if kind == "ct" else (0.02, 0.1, 0.1)
    for k, errs in run_pair(kind, 48, 60, 70, tv, lam, alpha, beta, iters=[1, 20], solver="pdhg"):
        for name, e in errs.items():
            assert e <= (2e-5 if k == 1 else 2e-4), (k, name, e)


def test_iterations_full_size_sampled():
    """512x512 workload geometry, 3 NCS iterations in the launch configuration the
    benchmark times; compared in full against the oracle (the oracle runs one
    512x512 iteration in about a second)."""
    for k, errs in run_pair("ct", 512, 720, 730, "iso", lam=0.005, alpha=1.0, beta=3.0, iters=[3]):
        for name, e in errs.items():
            assert e <= 1e-4, (k, name, e)


def test_pdhg_only_plan():
    """A pdhg_only plan (no M, no (A3) power iteration) runs the same PDHG iterates as a
    full plan, bit for bit, and refuses the entry points that need M."""
    import paper_1810_13100_gb300 as ncs
    N, na, nd = 64, 90, 92
    pr = synth.ct_problem(2, N, na, nd, 8, 0.01, oproj(N, na, nd))
    b = torch.from_numpy(pr["b"].ravel()).cuda()
    res = []
    for only in (False, True):
        plan = ncs.Plan(N, na, nd, 0.3, 1.0, beta=3.0, tv="iso", pdhg_only=only)
        x = torch.zeros(N * N, device="cuda")
        u = torch.zeros(na * nd, device="cuda")
        v = torch.zeros(2 * N * N, device="cuda")
        plan.pdhg_step(x, u, v, None, b, n_iter=15)
        torch.cuda.synchronize()
        res.append(to_np(x))
        if only:
            with pytest.raises(ncs.NCSError) as ei:
                plan.step(x, u, v, None, b, n_iter=1)
            assert ei.value.code == -2
            with pytest.raises(ncs.NCSError) as ei:
                plan.solve(b, x, tol=1e-4, max_iter=10)
            assert ei.value.code == -2
            with pytest.raises(ncs.NCSError):
                plan.apply_Minv(x)
            lm, rho = plan.power_bound()
            assert lm > 0 and np.isnan(rho)
        plan.close()
    assert np.array_equal(res[0], res[1])
