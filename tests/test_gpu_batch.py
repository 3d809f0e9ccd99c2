"""Batches of independent slices (ncs_batch_solve) and the plan autotuner.

A batch runs every slice's iterations as branches of one CUDA graph; each
slice's iterates must equal, bit for bit, those of the same plan solved alone
(the kernels and their order per slice are identical).  A batch solve to a gap
is checked by the FP64 oracle.  Autotuned plans (gather slicing, FFT radix
order) keep operator parity with the oracle."""
import json
import os

import numpy as np
import pytest

import synth
from helpers import f32, oproj, oracle_scaled_mu, rel_l2, to_np
from oracle import circulant as oci
from oracle import operators as oop
from oracle import solvers as osv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SLICES = [(48, 60, 70, "aniso", 3), (96, 140, 130, "iso", 4), (64, 90, 92, "aniso", 5), (384, 538, 386, "iso", 6)]


def make(N, na, nd, tv, seed, **kw):
    import paper_1810_13100_gb300 as ncs
    pr = synth.ct_problem(seed, N, na, nd, 8, 0.01, oproj(N, na, nd))
    plan = ncs.Plan(N, na, nd, 0.05, 0.01, beta=0.01, tv=tv, **kw)
    return plan, torch.from_numpy(pr["b"].ravel()).cuda()


def test_batch_iterates_equal_single_solves():
    import paper_1810_13100_gb300 as ncs
    made = [make(*s) for s in SLICES]
    plans = [m[0] for m in made]
    bs = [m[1] for m in made]
    xs = [torch.zeros(p.n, device="cuda") for p in plans]
    batch = ncs.Batch(plans)
    code, reps = batch.solve(bs, xs, tol=0.0, max_iter=35, f_stars=[-1e300] * len(plans))
    assert code == 1 and all(r["iters"] == 35 for r in reps)
    for p, b, xb in zip(plans, bs, xs):
        x1 = torch.zeros(p.n, device="cuda")
        rep = p.solve(b, x1, tol=0.0, max_iter=35, f_star=-1e300)
        torch.cuda.synchronize()
        assert rep["iters"] == 35
        assert torch.equal(x1, xb)
    batch.close()
    for p in plans:
        p.close()


def test_batch_lanes_keep_iterates_bitwise():
    """With 1 or 2 lanes (slices chained so fewer run at once) and with the tuned lane
    count, every slice's iterate after 35 iterations equals the all-concurrent one."""
    import paper_1810_13100_gb300 as ncs
    made = [make(*s) for s in SLICES + [(64, 90, 92, "iso", 7)]]
    plans = [m[0] for m in made]
    bs = [m[1] for m in made]
    batch = ncs.Batch(plans)
    ref = [torch.zeros(p.n, device="cuda") for p in plans]
    batch.solve(bs, ref, tol=0.0, max_iter=35, f_stars=[-1e300] * len(plans))
    for lanes in (1, 2, "tuned"):
        if lanes == "tuned":
            tmp = [torch.zeros(p.n, device="cuda") for p in plans]
            got = batch.tune_lanes(bs, tmp, iters=10)
            assert got in (0, 1, 2, 4)
        else:
            batch.set_lanes(lanes)
        xs = [torch.zeros(p.n, device="cuda") for p in plans]
        code, reps = batch.solve(bs, xs, tol=0.0, max_iter=35, f_stars=[-1e300] * len(plans))
        torch.cuda.synchronize()
        assert all(r["iters"] == 35 for r in reps)
        assert all(torch.equal(a, c) for a, c in zip(xs, ref)), lanes
    with pytest.raises(ncs.NCSError):
        batch.set_lanes(-1)
    batch.close()
    for p in plans:
        p.close()


def test_batch_solve_to_gap_checked_by_oracle():
    import paper_1810_13100_gb300 as ncs
    W = synth.WORKLOADS["ct64"]
    pr = synth.ct_problem(0, W["N"], W["n_angles"], W["n_det"], W["n_ellipses"], W["noise_frac"],
                          oproj(W["N"], W["n_angles"], W["n_det"]))
    with open(os.path.join(ROOT, "tests", "golden", "fstar_ct64_s0.json")) as fh:
        fs = json.load(fh)["f_star"]
    p0 = ncs.Plan(W["N"], W["n_angles"], W["n_det"], W["lam"], 0.01, beta=0.01, tv=W["tv"])
    b0 = torch.from_numpy(pr["b"].ravel()).cuda()
    p1, b1 = make(96, 140, 130, "iso", 4)
    x0 = torch.zeros(p0.n, device="cuda")
    x1 = torch.zeros(p1.n, device="cuda")
    batch = ncs.Batch([p0, p1])
    code, reps = batch.solve([b0, b1], [x0, x1], tol=1e-4, max_iter=20000, f_stars=[fs, None])
    assert code == 0 and reps[0]["status"] == 0 and reps[1]["status"] == 0
    assert reps[0]["gap"] <= 1e-4
    g = oop.Geometry(W["N"], W["n_angles"], W["n_det"])
    P = osv.Problem(g, f32(pr["b"]), lam=W["lam"], alpha=0.01, beta=0.01, tv=W["tv"])
    f_oracle = osv.objective(P, to_np(x0).reshape(W["N"], W["N"]))
    assert f_oracle <= fs * (1 + 1e-4 + 1e-6)
    batch.close()
    p0.close()
    p1.close()


@pytest.mark.parametrize("N,na,nd", [(96, 140, 130), (384, 538, 386), (512, 720, 730)])
def test_autotuned_plan_keeps_parity(N, na, nd):
    import paper_1810_13100_gb300 as ncs
    plan = ncs.Plan(N, na, nd, 0.01, 1.0, beta=3.0, tv="iso", autotune=True, power_tol=1e-9)
    info = plan.info()
    assert info["gather_parts"] >= 1 and int(np.prod(info["fft_radices"])) == N
    g = oop.Geometry(N, na, nd)
    rng = np.random.default_rng(N)
    yv = f32(rng.uniform(-1, 1, (na, nd)))
    xt = plan.apply_KT(torch.from_numpy(yv.ravel().astype(np.float32)).cuda())
    assert rel_l2(to_np(xt), oop.KT(yv, g)) <= 1e-5
    mu_ref, _ = oracle_scaled_mu(N, na, nd, 1.0, 3.0, 0.0, "iso")
    r = f32(rng.standard_normal((N, N)))
    out = plan.apply_Minv(torch.from_numpy(r.ravel().astype(np.float32)).cuda())
    assert rel_l2(to_np(out), oci.circulant_solve(r, mu_ref)) <= 1e-5
    plan.close()
