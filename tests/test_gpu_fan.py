"""GPU parity of the fan-beam path (Sec. 4, fan beam geometry: the divergent-beam transform
with an equiangular detector), through the C ABI, against the FP64 oracle's fan-beam Joseph
projector (oracle/operators.py FanGeometry, itself pinned in tests/test_oracle_fan.py) on the
same seeded FP32 inputs.

Tolerances are those of the parallel beam (tests/test_gpu_operators.py and
tests/test_gpu_iterations.py): relative L2 <= 1e-5 per operator, 2e-5 after one NCS / PDHG
iteration and 2e-4 after 20.  The forward kernel evaluates the crossings from the same split
FP32 coefficients as the parallel beam (per ray instead of per angle), and the pixel-driven
gather evaluates the identical weights, so the GPU pair is an exact transpose up to the FP32
summation order."""
import json
import math
import os

import numpy as np
import pytest

import synth
from helpers import f32, rel_l2, to_np, v_to_oracle
from oracle import circulant as oci
from oracle import operators as oop
from oracle import solvers as osv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TOL = 1e-5

USER_VIEWS = [0.1, 0.7, 1.3, 2.0, 3.3, 4.4, 5.9]

# (N, n_views, n_det, R, pitch, offset, views): tiny and full sizes, ragged 32 x 8 pixel
# blocks and 64-channel tiles, a shifted detector, a narrow fan pitch (many rays per pixel
# and view), user source angles
FAN_GEOMS = [
    (8, 12, 16, 9.0, synth.fan_pitch(8, 9.0, 16, 1.05), 0.0, None),
    (48, 60, 70, 60.0, synth.fan_pitch(48, 60.0, 70, 1.05), 0.0, None),
    (64, 120, 96, 128.0, synth.fan_pitch(64, 128.0, 96, 1.05), 0.0, None),
    (96, 90, 130, 100.0, synth.fan_pitch(96, 100.0, 130, 1.05), 0.37 * synth.fan_pitch(96, 100.0, 130, 1.05), None),
    (32, 7, 300, 25.0, 0.004, 0.0, USER_VIEWS),
    (512, 720, 768, 1024.0, synth.fan_pitch(512, 1024.0, 768, 1.02), 0.0, None),
]


def fan_plan(N, na, nd, R, pitch, off, views, **kw):
    import paper_1810_13100_gb300 as ncs
    lam = kw.pop("lam", 0.01)
    alpha = kw.pop("alpha", 1.0)
    return ncs.Plan(N, na, nd, lam, alpha, src_dist=R, fan_pitch=pitch, fan_offset=off, angles=views, **kw)


def ogeom(N, na, nd, R, pitch, off, views):
    return oop.FanGeometry(N, na, nd, R, pitch, off, beta=None if views is None else np.asarray(views))


@pytest.mark.parametrize("N,na,nd,R,pitch,off,views", FAN_GEOMS)
def test_fan_forward_parity(N, na, nd, R, pitch, off, views):
    x = f32(np.random.default_rng(N + na).uniform(-1, 1, (N, N)))
    ref = oop.K(x, ogeom(N, na, nd, R, pitch, off, views))
    plan = fan_plan(N, na, nd, R, pitch, off, views, power_max_iter=2, h_probes=1)
    y = plan.apply_K(torch.from_numpy(x.ravel().astype(np.float32)).cuda())
    plan.close()
    assert rel_l2(to_np(y), ref) <= TOL


@pytest.mark.parametrize("kernel", ["lines", "quads"])
@pytest.mark.parametrize("N,na,nd,R,pitch,off,views", FAN_GEOMS)
def test_fan_gather_transpose_parity(N, na, nd, R, pitch, off, views, kernel):
    """Both K^T kernels: the ray-driven tile walk (default) and the pixel-driven quads."""
    yv = f32(np.random.default_rng(7 * N + na).uniform(-1, 1, (na, nd)))
    ref = oop.KT(yv, ogeom(N, na, nd, R, pitch, off, views))
    plan = fan_plan(N, na, nd, R, pitch, off, views, power_max_iter=2, h_probes=1, fan_gather=kernel)
    x = plan.apply_KT(torch.from_numpy(yv.ravel().astype(np.float32)).cuda())
    plan.close()
    assert rel_l2(to_np(x), ref) <= TOL


@pytest.mark.parametrize("kernel", ["lines", "quads"])
@pytest.mark.parametrize("N,na,nd,R,pitch,off,views", FAN_GEOMS[:5])
def test_fan_gpu_pair_is_exact_transpose(N, na, nd, R, pitch, off, views, kernel):
    """<K x, y> = <x, K^T y> for the GPU pair (FP64 dot products of the FP32 results)."""
    plan = fan_plan(N, na, nd, R, pitch, off, views, power_max_iter=2, h_probes=1, fan_gather=kernel)
    gen = torch.Generator(device="cuda").manual_seed(5)
    for _ in range(3):
        x = torch.rand(N * N, device="cuda", generator=gen) * 2 - 1
        y = torch.rand(na * nd, device="cuda", generator=gen) * 2 - 1
        lhs = float(torch.dot(plan.apply_K(x).double(), y.double()))
        rhs = float(torch.dot(x.double(), plan.apply_KT(y).double()))
        scale = float(torch.dot(plan.apply_K(x.abs()).double(), y.abs().double()))
        assert abs(lhs - rhs) <= 1e-6 * scale
    plan.close()


@pytest.mark.parametrize("kernel", ["lines", "quads"])
@pytest.mark.parametrize("N,na,nd,R,pitch", [(4096, 6, 4100, 8192.0, synth.fan_pitch(4096, 8192.0, 4100, 1.02)),
                                             (16, 1, 1, 20.0, 0.05), (12, 3, 2, 15.0, 0.3)])
def test_fan_extreme_sizes_parity(N, na, nd, R, pitch, kernel):
    """The largest image side, a single ray, and a fan of two channels wider than the image."""
    rng = np.random.default_rng(N + 5 * na)
    x = f32(rng.uniform(-1, 1, (N, N)))
    yv = f32(rng.uniform(-1, 1, (na, nd)))
    g = ogeom(N, na, nd, R, pitch, 0.0, None)
    plan = fan_plan(N, na, nd, R, pitch, 0.0, None, power_max_iter=2, h_probes=1, fan_gather=kernel)
    y = plan.apply_K(torch.from_numpy(x.ravel().astype(np.float32)).cuda())
    ref = oop.K(x, g)
    assert rel_l2(to_np(y), ref) <= TOL
    xt = plan.apply_KT(torch.from_numpy(yv.ravel().astype(np.float32)).cuda())
    assert rel_l2(to_np(xt), oop.KT(yv, g)) <= TOL
    plan.close()


def oracle_fan_mu(g, alpha, beta, probes, gamma=0.0):
    """The oracle's eigenvalues of M for a fan plan before the (A3) rescale: eq. (H-fan) in
    least-squares form over the plan's float32 SplitMix64 probes, DC ||K 1||^2 / ||1||^2."""
    N = g.N
    vs = [f32(osv.splitmix64_uniform(1 + q, N * N)).reshape(N, N) for q in range(probes)]
    h = np.maximum(oci.probe_ls(lambda v: oop.KT(oop.K(v, g), g), N, vs), 0.0)
    h[0, 0] = oci.h_dc_default(g)
    return gamma + alpha * h + (beta * beta / alpha) * oci.H_D(N)


def test_fan_probe_mu_matches_oracle():
    N, na, nd, R = 48, 60, 70, 60.0
    pitch = synth.fan_pitch(N, R, nd, 1.05)
    alpha, beta, P = 0.5, 1.5, 4
    plan = fan_plan(N, na, nd, R, pitch, 0.0, None, lam=0.01, alpha=alpha, beta=beta, h_probes=P,
                    a3_margin=-1.0, power_max_iter=2)
    mu_gpu = plan.mu()
    plan.close()
    mu_ref = oracle_fan_mu(ogeom(N, na, nd, R, pitch, 0.0, None), alpha, beta, P)
    assert rel_l2(mu_gpu, mu_ref) <= 1e-4


def run_fan_pair(N, na, nd, R, pitch, tv, lam, alpha, beta, iters, solver="ncs", probes=8, kernel="auto"):
    import paper_1810_13100_gb300 as ncs
    g = ogeom(N, na, nd, R, pitch, 0.0, None)
    pr = synth.ct_problem(1, N, na, nd, 8, 0.01, lambda x: oop.K(x, g))
    P = osv.Problem(g, f32(pr["b"]), lam=lam, alpha=alpha, beta=beta, tv=tv)
    plan = ncs.Plan(N, na, nd, lam, alpha, beta=beta, tv=tv, src_dist=R, fan_pitch=pitch, h_probes=probes,
                    fan_gather=kernel, power_tol=1e-9)
    b = torch.from_numpy(pr["b"].ravel()).cuda()
    x = torch.zeros(N * N, device="cuda")
    u = torch.zeros(na * nd, device="cuda")
    v = torch.zeros(2 * N * N, device="cuda")
    st = osv.zero_state(P)
    if solver == "ncs":
        mus, _ = osv.a3_scaled_mu(P, oracle_fan_mu(g, alpha, beta, probes))
        Minv = osv.circulant_Minv(mus)
        step = lambda s_: osv.ncs_step(P, s_, Minv)
        gpu_step = plan.step
    else:
        gp, _ = osv.pdhg_gamma(P)
        step = lambda s_: osv.pdhg_step(P, s_, gp)
        gpu_step = plan.pdhg_step
    out, done = [], 0
    for k in iters:
        gpu_step(x, u, v, None, b, None, n_iter=k - done)
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
        out.append((k, dict(x=rel_l2(to_np(x), st.x), u=rel_l2(to_np(u), st.u),
                            v=np.linalg.norm(np.concatenate([vh.ravel(), vv.ravel()]) - vref) / max(vscale, 1e-300))))
    plan.close()
    return out


@pytest.mark.parametrize("solver,tv,kernel", [("ncs", "aniso", "lines"), ("ncs", "iso", "lines"),
                                              ("pdhg", "iso", "lines"), ("ncs", "iso", "quads"),
                                              ("pdhg", "aniso", "quads")])
def test_fan_iterations(solver, tv, kernel):
    N, na, nd, R = 48, 60, 70, 60.0
    pitch = synth.fan_pitch(N, R, nd, 1.05)
    for k, errs in run_fan_pair(N, na, nd, R, pitch, tv, 0.3, 1.0, 3.0, [1, 5, 20], solver=solver, kernel=kernel):
        for name, e in errs.items():
            assert e <= (2e-5 if k == 1 else 2e-4), (k, name, e)


def test_fan_solve_reaches_gap_checked_by_oracle():
    """ncs_solve on the 64x64 fan-beam workload (120 views, 96 channels, source at 128 pixels)
    from zero to the 1e-4 relative gap against the oracle's f* (tests/golden/fstar_fan64_s0.json),
    then the oracle's FP64 objective of the returned image."""
    import paper_1810_13100_gb300 as ncs
    W = synth.WORKLOADS["fan64"]
    with open(os.path.join(ROOT, "tests", "golden", "fstar_fan64_s0.json")) as fh:
        fs = json.load(fh)["f_star"]
    N, na, nd = W["N"], W["n_angles"], W["n_det"]
    pitch = synth.fan_pitch(N, W["src_dist"], nd, W["cover"])
    g = oop.FanGeometry(N, na, nd, W["src_dist"], pitch)
    pr = synth.ct_problem(0, N, na, nd, W["n_ellipses"], W["noise_frac"], lambda x: oop.K(x, g))
    P = osv.Problem(g, f32(pr["b"]), lam=W["lam"], alpha=0.01, beta=0.01, tv=W["tv"])
    plan = ncs.Plan(N, na, nd, W["lam"], 0.01, beta=0.01, tv=W["tv"], src_dist=W["src_dist"], fan_pitch=pitch)
    b = torch.from_numpy(pr["b"].ravel()).cuda()
    x = torch.zeros(N * N, device="cuda")
    rep = plan.solve(b, x, tol=1e-4, max_iter=20000, f_star=fs)
    plan.close()
    assert rep["status"] == 0, rep
    f_oracle = osv.objective(P, x.double().cpu().numpy().reshape(N, N))
    assert f_oracle <= fs * (1 + 1e-4 + 1e-6)
    assert f_oracle >= fs * (1 - 1e-6)
    assert rep["f"] == pytest.approx(f_oracle, rel=1e-6)


def test_fan_kernels_agree_and_autotune_keeps_one():
    """The two K^T kernels give the same image up to FP32 summation order, and a plan with the
    autotuner (which times both) still matches them."""
    N, na, nd, R = 96, 90, 130, 100.0
    pitch = synth.fan_pitch(N, R, nd, 1.05)
    yv = torch.from_numpy(f32(np.random.default_rng(2).uniform(-1, 1, (na, nd))).ravel().astype(np.float32)).cuda()
    outs = []
    for kernel, tune in (("lines", False), ("quads", False), ("auto", True)):
        plan = fan_plan(N, na, nd, R, pitch, 0.0, None, power_max_iter=2, h_probes=1, fan_gather=kernel,
                        autotune=tune)
        outs.append(to_np(plan.apply_KT(yv)))
        plan.close()
    assert rel_l2(outs[0], outs[1]) <= 2e-6
    assert min(rel_l2(outs[2], outs[0]), rel_l2(outs[2], outs[1])) <= 2e-6


def test_fan_fbp_is_unsupported():
    import paper_1810_13100_gb300 as ncs
    N, na, nd, R = 32, 24, 48, 40.0
    plan = fan_plan(N, na, nd, R, synth.fan_pitch(N, R, nd, 1.05), 0.0, None, power_max_iter=2, h_probes=1)
    with pytest.raises(ncs.NCSError):
        plan.fbp(torch.zeros(na * nd, device="cuda"))
    plan.close()


def test_fan_and_parallel_plans_in_one_batch_equal_single_solves():
    """Fan-beam plans (both K^T kernels) and a parallel-beam plan solved together by
    ncs_batch_solve give, bit for bit, the iterates of each plan solved alone."""
    import paper_1810_13100_gb300 as ncs
    specs = [(48, 60, 70, 60.0, "lines"), (64, 120, 96, 128.0, "quads"), (96, 90, 130, 100.0, "lines")]
    plans, bs = [], []
    for k, (N, na, nd, R, kern) in enumerate(specs):
        pitch = synth.fan_pitch(N, R, nd, 1.05)
        g = oop.FanGeometry(N, na, nd, R, pitch)
        pr = synth.ct_problem(10 + k, N, na, nd, 8, 0.01, lambda x, g=g: oop.K(x, g))
        plans.append(ncs.Plan(N, na, nd, 0.05, 0.01, tv="iso", src_dist=R, fan_pitch=pitch, h_probes=8,
                              fan_gather=kern))
        bs.append(torch.from_numpy(pr["b"].ravel()).cuda())
    pr = synth.ct_problem(13, 64, 90, 92, 8, 0.01, lambda x: oop.K(x, oop.Geometry(64, 90, 92)))
    plans.append(ncs.Plan(64, 90, 92, 0.05, 0.01, tv="aniso"))
    bs.append(torch.from_numpy(pr["b"].ravel()).cuda())
    xs = [torch.zeros(p.n, device="cuda") for p in plans]
    batch = ncs.Batch(plans)
    code, reps = batch.solve(bs, xs, tol=0.0, max_iter=25, f_stars=[-1e300] * len(plans))
    assert code == 1 and all(r["iters"] == 25 for r in reps)
    for p, b, xb in zip(plans, bs, xs):
        x1 = torch.zeros(p.n, device="cuda")
        rep = p.solve(b, x1, tol=0.0, max_iter=25, f_star=-1e300)
        torch.cuda.synchronize()
        assert rep["iters"] == 25
        assert torch.equal(x1, xb)
    batch.close()
    for p in plans:
        p.close()


@pytest.mark.parametrize("kernel", ["lines", "quads"])
def test_fan_bf16_iterations_against_oracle(kernel):
    """BF16 storage of the duals and the projector's images on a fan plan (both K^T kernels):
    x against the oracle within the bfloat16 bounds of tests/test_gpu_bf16.py (4e-3 after one
    iteration, 2e-2 after 20)."""
    import paper_1810_13100_gb300 as ncs
    N, na, nd, R = 48, 60, 70, 60.0
    pitch = synth.fan_pitch(N, R, nd, 1.05)
    lam, alpha, beta, probes = 0.3, 1.0, 3.0, 8
    g = ogeom(N, na, nd, R, pitch, 0.0, None)
    pr = synth.ct_problem(2, N, na, nd, 8, 0.01, lambda x: oop.K(x, g))
    P = osv.Problem(g, f32(pr["b"]), lam=lam, alpha=alpha, beta=beta, tv="iso")
    plan = ncs.Plan(N, na, nd, lam, alpha, beta=beta, tv="iso", src_dist=R, fan_pitch=pitch, h_probes=probes,
                    precision="bf16", fan_gather=kernel, power_tol=1e-9)
    mus, _ = osv.a3_scaled_mu(P, oracle_fan_mu(g, alpha, beta, probes))
    Minv = osv.circulant_Minv(mus)
    b = torch.from_numpy(pr["b"].ravel()).cuda()
    x = torch.zeros(N * N, device="cuda")
    u = torch.zeros(na * nd, device="cuda", dtype=torch.bfloat16)
    v = torch.zeros(2 * N * N, device="cuda", dtype=torch.bfloat16)
    st, done = osv.zero_state(P), 0
    for k, tol in ((1, 4e-3), (20, 2e-2)):
        plan.step(x, u, v, None, b, None, n_iter=k - done)
        for _ in range(k - done):
            st = osv.ncs_step(P, st, Minv)
        done = k
        torch.cuda.synchronize()
        assert rel_l2(to_np(x), st.x) <= tol, (k, "x")
        assert rel_l2(to_np(u.float()), st.u) <= tol, (k, "u")
    plan.close()


def test_fan_admm_iterates_match_oracle():
    """The ADMM comparator (admm_solve) on a fan plan against the oracle's admm_pcg with the
    same probe-estimated M (tolerances of tests/test_gpu_admm.py: 2e-4 after one outer step,
    2e-3 after five)."""
    import paper_1810_13100_gb300 as ncs
    N, na, nd, R = 48, 60, 70, 60.0
    pitch = synth.fan_pitch(N, R, nd, 1.05)
    lam, a, n_cg, probes = 0.01, 0.1, 3, 8
    g = ogeom(N, na, nd, R, pitch, 0.0, None)
    pr = synth.ct_problem(0, N, na, nd, 8, 0.01, lambda x: oop.K(x, g))
    P = osv.Problem(g, f32(pr["b"]), lam=lam, alpha=a, beta=a, tv="iso")
    mus, _ = osv.a3_scaled_mu(P, oracle_fan_mu(g, a, a, probes))
    xs = osv.admm_pcg(P, 5, n_cg, osv.circulant_Minv(mus))
    plan = ncs.Plan(N, na, nd, lam, a, beta=a, tv="iso", src_dist=R, fan_pitch=pitch, h_probes=probes,
                    power_tol=1e-9)
    b = torch.from_numpy(pr["b"].ravel()).cuda()
    x = torch.zeros(N * N, device="cuda")
    for k, tol in ((1, 2e-4), (5, 2e-3)):
        x.zero_()
        rep = plan.admm_solve(b, x, tol=0.0, max_outer=k, n_cg=n_cg)
        assert rep["iters"] == k
        assert rel_l2(to_np(x), xs[k - 1]) <= tol, k
    plan.close()
