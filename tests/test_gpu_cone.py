"""GPU parity of the cone-beam operator pair (ncs_cone_apply_K / _KT; Sec. 4, cone beam
geometry), through the C ABI, against the FP64 oracle's cone-beam Joseph projector
(oracle/cone.py, pinned in tests/test_oracle_cone.py) on the same seeded FP32 inputs.

Tolerance: relative L2 <= 1e-5, as for the 2-D projectors: the in-plane weights come from the
fan beam's split FP32 coefficients and the slice coordinate is evaluated in FP64, so each tap
weight is within ~1e-7 and the FP32 sums add sqrt(4N) * 6e-8.  The transpose is a gather over
2 x 2 pixel quads of one slice that evaluates the forward's weights, so the GPU pair is adjoint
up to the FP32 summation order."""
import math

import numpy as np
import pytest

from helpers import f32, rel_l2, to_np
from oracle import cone as oc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5
VIEWS = [0.1, 0.7, 1.3, 2.0, 3.3, 4.4, 5.9]


def cover(N, R, nd, slack=1.05):
    return 2.0 * math.asin(N / math.sqrt(2.0) / R) / nd * slack


# (N, Nz, views, rows, channels, R, pitch, row pitch, offset, row offset, source angles)
GEOMS = [
    (16, 8, 10, 6, 24, 20.0, cover(16, 20.0, 24), 0.1, 0.0, 0.0, None),
    (48, 10, 12, 9, 64, 60.0, cover(48, 60.0, 64), 0.04, 0.004, 0.005, None),   # ragged tiles, offsets
    (32, 6, 7, 5, 40, 25.0, 0.03, 0.12, 0.0, 0.0, VIEWS),                       # wide fan, user views
    (24, 1, 8, 3, 30, 40.0, cover(24, 40.0, 30), 0.02, 0.0, 0.0, None),         # a single slice
    (64, 16, 16, 16, 96, 128.0, cover(64, 128.0, 96), 0.01, 0.0, 0.0, None),
]


def make(N, Nz, na, nr, nd, R, pitch, rp, off, roff, views):
    import paper_1810_13100_gb300 as ncs
    cone = ncs.Cone(N, Nz, na, nr, nd, R, pitch, rp, offset=off, row_offset=roff, views=views)
    g = oc.ConeGeometry(N, Nz, na, nr, nd, R, pitch, rp, off, roff, beta=None if views is None else np.array(views))
    return cone, g


@pytest.mark.parametrize("geom", GEOMS)
def test_cone_forward_parity(geom):
    cone, g = make(*geom)
    x = f32(np.random.default_rng(geom[0] + geom[1]).uniform(-1, 1, g.shape))
    y = cone.apply_K(torch.from_numpy(x.ravel().astype(np.float32)).cuda())
    cone.close()
    assert rel_l2(to_np(y), oc.K(x, g)) <= TOL


@pytest.mark.parametrize("geom", GEOMS)
def test_cone_transpose_parity(geom):
    cone, g = make(*geom)
    yv = f32(np.random.default_rng(7 * geom[0] + geom[2]).uniform(-1, 1, g.sino_shape))
    x = cone.apply_KT(torch.from_numpy(yv.ravel().astype(np.float32)).cuda())
    cone.close()
    assert rel_l2(to_np(x), oc.KT(yv, g)) <= TOL


@pytest.mark.parametrize("geom", GEOMS[:3])
def test_cone_gpu_pair_is_adjoint(geom):
    cone, g = make(*geom)
    gen = torch.Generator(device="cuda").manual_seed(11)
    for _ in range(2):
        x = torch.rand(g.n, device="cuda", generator=gen) * 2 - 1
        y = torch.rand(g.m, device="cuda", generator=gen) * 2 - 1
        lhs = float(torch.dot(cone.apply_K(x).double(), y.double()))
        rhs = float(torch.dot(x.double(), cone.apply_KT(y).double()))
        scale = float(torch.dot(cone.apply_K(x.abs()).double(), y.abs().double()))
        assert abs(lhs - rhs) <= 1e-6 * scale
    cone.close()


def test_cone_rejects_steep_rows_and_a_close_source():
    import paper_1810_13100_gb300 as ncs
    with pytest.raises(ncs.NCSError):
        ncs.Cone(16, 4, 4, 5, 8, 20.0, 0.05, 0.4)            # outer rows' slopes +-0.8 > 1/sqrt(2)
    with pytest.raises(ncs.NCSError):
        ncs.Cone(16, 4, 4, 3, 8, 12.0, 0.05, 0.1)            # source inside the circle plus 3 pixels


# ---------------------------------------------------------------- the 3-D NCS iteration

# 32 x 32 x 8 volume, 12 views on a full turn, 8 rows x 48 channels, source at 40 voxels
NG = (32, 8, 12, 8, 48, 40.0)


def nplan(ncs, lam, alpha, tv, **kw):
    N, Nz, na, nr, nd, R = NG
    return ncs.ConePlan(N, Nz, na, nr, nd, R, cover(N, R, nd), 0.08, lam, alpha, tv=tv, **kw)


def oproblem(lam, alpha, tv, seed=0):
    import synth
    N, Nz, na, nr, nd, R = NG
    g = oc.ConeGeometry(N, Nz, na, nr, nd, R, cover(N, R, nd), 0.08)
    pr = synth.ct3d_problem(seed, N, Nz, na, nr, nd, 6, 0.01, lambda x: oc.K(x, g))
    P = oc.Problem(g, pr["b"].astype(np.float64), lam=lam, alpha=alpha, beta=alpha, tv=tv)
    return g, pr, P


def test_cone_mu_and_solve_match_oracle():
    """M's eigenvalues before the (A3) rescale (eq. (H-fan) over 4 probe volumes, the 3-D
    Laplacian spectrum) against the oracle's mu_probes, and the 3-D FFT solve against the
    oracle's circulant solve with the same eigenvalues."""
    import paper_1810_13100_gb300 as ncs
    g, pr, P = oproblem(0.01, 0.5, "iso")
    plan = nplan(ncs, 0.01, 0.5, "iso", h_probes=4, a3_margin=-1.0, power_max_iter=2)
    mu_gpu = plan.mu()
    mu_ref = oc.mu_probes(P, 4)
    err = rel_l2(mu_gpu, mu_ref)
    print("cone mu rel L2 %.2e" % err)
    assert err <= 1e-4
    r = f32(np.random.default_rng(5).standard_normal(g.shape))
    out = plan.apply_Minv(torch.from_numpy(r.ravel().astype(np.float32)).cuda())
    assert rel_l2(to_np(out), oc.circulant_solve(r, mu_gpu)) <= 1e-5
    plan.close()


def test_cone_rho_and_objective_match_oracle():
    import paper_1810_13100_gb300 as ncs
    g, pr, P = oproblem(0.01, 0.5, "iso")
    plan = nplan(ncs, 0.01, 0.5, "iso", h_probes=4, power_tol=1e-9)
    _, rho_ref = oc.a3_scaled_mu(P, oc.mu_probes(P, 4))
    assert plan.power_bound() == pytest.approx(rho_ref, rel=1e-5)
    x = f32(pr["x_true"] + 0.05 * np.random.default_rng(1).standard_normal(g.shape))
    f = plan.objective(torch.from_numpy(x.ravel().astype(np.float32)).cuda(), torch.from_numpy(pr["b"].ravel()).cuda())
    assert f == pytest.approx(oc.objective(P, x), rel=1e-6)
    plan.close()


@pytest.mark.parametrize("tv", ["aniso", "iso"])
def test_cone_ncs_iterations_match_oracle(tv):
    """Whole 3-D NCS iterations (gather with D^T, 3-D FFT solve, forward with the data prox,
    3-D TV prox) from zero against the oracle's: 2e-5 after one iteration, 2e-4 after 20 (the
    TV dual against the size of its projection's argument, as for the 2-D iterations)."""
    import paper_1810_13100_gb300 as ncs
    lam, alpha = 0.05, 0.5
    g, pr, P = oproblem(lam, alpha, tv)
    plan = nplan(ncs, lam, alpha, tv, h_probes=4, power_tol=1e-9)
    mus, _ = oc.a3_scaled_mu(P, oc.mu_probes(P, 4))
    Minv = lambda r: oc.circulant_solve(r, mus)
    b = torch.from_numpy(pr["b"].ravel()).cuda()
    x = torch.zeros(g.n, device="cuda")
    u = torch.zeros(g.m, device="cuda")
    v = torch.zeros(3 * g.n, device="cuda")
    st = oc.zero_state(P)
    done = 0
    for k, tol in ((1, 2e-5), (20, 2e-4)):
        plan.step(x, u, v, b, n_iter=k - done)
        prev = st
        for _ in range(k - done):
            prev = st
            st = oc.ncs_step(P, st, Minv)
        done = k
        torch.cuda.synchronize()
        Nz, N = g.Nz, g.N
        vg = to_np(v).reshape(3, Nz, N, N)
        vgpu = np.concatenate([vg[0][:, :, :-1].ravel(), vg[1][:, :-1, :].ravel(), vg[2][:-1, :, :].ravel()])
        vref = np.concatenate([c.ravel() for c in st.v])
        dref = oc.D(2.0 * st.x - prev.x)
        vscale = np.linalg.norm(vref) + P.beta * np.sqrt(sum(np.sum(d * d) for d in dref))
        ex, eu = rel_l2(to_np(x), st.x), rel_l2(to_np(u), st.u)
        ev = np.linalg.norm(vgpu - vref) / max(vscale, 1e-300)
        print("cone %s after %d: x %.2e u %.2e v %.2e" % (tv, k, ex, eu, ev))
        assert ex <= tol and eu <= tol and ev <= tol, (k, ex, eu, ev)
        # the padding of the dual blocks stays zero
        assert not vg[0][:, :, -1].any() and not vg[1][:, -1, :].any() and not vg[2][-1].any()
    plan.close()


def test_cone_solve_reaches_gap_checked_by_oracle():
    """A 3-D NCS solve from zero to the 1e-4 gap against a reference minimum that the FP64
    oracle computes here (4000 iterations at the fastest step of the {1,3} x 10^p grid, whose
    last 1000 lower f by less than 1e-6 relative, 1% of the tolerance); the oracle's f(x_gpu)
    is then within 1e-4 of it."""
    import paper_1810_13100_gb300 as ncs
    lam, alpha = 0.01, 0.02
    g, pr, P = oproblem(lam, alpha, "iso", seed=2)
    mus, _ = oc.a3_scaled_mu(P, oc.mu_probes(P, 8))
    Minv = lambda r: oc.circulant_solve(r, mus)
    st = oc.run(P, oc.zero_state(P), 3000, Minv)
    f3000 = oc.objective(P, st.x)
    st = oc.run(P, st, 1000, Minv)
    fs = oc.objective(P, st.x)
    assert f3000 - fs <= 1e-6 * fs
    plan = nplan(ncs, lam, alpha, "iso", h_probes=8)
    b = torch.from_numpy(pr["b"].ravel()).cuda()
    x = torch.zeros(g.n, device="cuda")
    rep = plan.solve(b, x, tol=0.98e-4, max_iter=4000, f_star=fs)
    plan.close()
    assert rep["status"] == 0, rep
    f = oc.objective(P, to_np(x).reshape(g.shape))
    print("cone solve: %d iterations, %.1f ms, oracle gap %.3e" % (rep["iters"], rep["time_ms"], (f - fs) / fs))
    assert fs * (1 - 1e-7) <= f <= fs * (1 + 1e-4)


def test_cone_plan_counts_its_kernels():
    """ncs_cone_kernels: an NCS step enqueues 8 kernels (the gather, five of the 3-D circulant
    solve, the forward pass with the data prox, the TV prox) and an objective 3."""
    import paper_1810_13100_gb300 as ncs
    g, pr, _ = oproblem(0.01, 0.02, "iso")
    plan = nplan(ncs, 0.01, 0.02, "iso", h_probes=4)
    b = torch.from_numpy(pr["b"].ravel()).cuda()
    x = torch.zeros(g.n, device="cuda")
    u = torch.zeros(b.numel(), device="cuda")
    v = torch.zeros(3 * g.n, device="cuda")
    k0 = plan.kernels()
    plan.step(x, u, v, b, n_iter=3)
    assert plan.kernels() - k0 == 24
    k1 = plan.kernels()
    plan.objective(x, b)
    assert plan.kernels() - k1 == 3
    plan.close()
