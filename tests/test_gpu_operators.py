"""GPU parity of the operators, through the C ABI, against the FP64 oracle on
the same seeded FP32 inputs.

Tolerance: relative L2 <= 1e-5 per operator in FP32.  Derivation: the
projector sums <= 2N FP32 taps per ray with FP32 interpolation weights whose
rounding (|f| < 2N, one ulp ~ 2N * 6e-8) changes a tap by ~1e-5 of a pixel
difference; over a ray these errors average out to ~1e-6 relative, and the
FP32 accumulation adds sqrt(2N) * 6e-8 ~ 2e-6.  The FFT solve carries
log2(N) FP32 butterflies (~1e-6)."""
import math

import numpy as np
import pytest

from helpers import f32, oproj, oracle_scaled_mu, rel_l2, to_np, v_from_oracle, v_to_oracle
from oracle import circulant as oci
from oracle import operators as oop
from oracle import solvers as osv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5

# (N, n_angles, n_det, spacing, offset): several tiles plus ragged tails,
# tiny and full sizes, angle counts with and without exact pi/4 ties
GEOMS = [
    (8, 5, 11, 1.0, 0.0),          # smallest image, single partial tiles
    (48, 60, 70, 1.0, 0.0),        # ragged 32-pixel tiles, ragged 64-bin tile
    (64, 90, 92, 1.0, 0.0),        # 64x64 workload
    (96, 140, 130, 1.0, 0.0),
    (96, 36, 101, 1.5, 0.25),      # pitch > 1 and a shifted detector
    (384, 64, 386, 1.0, 0.0),      # radix-3 image side
    (512, 720, 730, 1.0, 0.0),     # 512x512 workload geometry (full size)
]


def plan_for(N, na, nd, sp=1.0, off=0.0, **kw):
    import paper_1810_13100_gb300 as ncs
    kw.setdefault("lam", 0.01)
    kw.setdefault("alpha", 1.0)
    lam = kw.pop("lam")
    alpha = kw.pop("alpha")
    return ncs.Plan(N, na, nd, lam, alpha, det_spacing=sp, det_offset=off, **kw)


@pytest.mark.parametrize("N,na,nd,sp,off", GEOMS)
def test_forward_projection_parity(N, na, nd, sp, off):
    rng = np.random.default_rng(N + na)
    x = f32(rng.uniform(-1, 1, (N, N)))
    g = oop.Geometry(N, na, nd, spacing=sp, offset=off)
    ref = oop.K(x, g)
    plan = plan_for(N, na, nd, sp, off, power_max_iter=2)
    y = plan.apply_K(torch.from_numpy(x.ravel().astype(np.float32)).cuda())
    assert rel_l2(to_np(y), ref) <= TOL


@pytest.mark.parametrize("N,na,nd,sp,off", GEOMS)
def test_gather_transpose_parity(N, na, nd, sp, off):
    rng = np.random.default_rng(7 * N + na)
    yv = f32(rng.uniform(-1, 1, (na, nd)))
    g = oop.Geometry(N, na, nd, spacing=sp, offset=off)
    ref = oop.KT(yv, g)
    plan = plan_for(N, na, nd, sp, off, power_max_iter=2)
    x = plan.apply_KT(torch.from_numpy(yv.ravel().astype(np.float32)).cuda())
    assert rel_l2(to_np(x), ref) <= TOL


@pytest.mark.parametrize("N,na,nd,sp,off", GEOMS[:5])
def test_gpu_pair_is_exact_transpose(N, na, nd, sp, off):
    """<K x, y> = <x, K^T y> for the GPU pair: both kernels evaluate the same
    FP32 weights, so only the FP32 accumulation order differs."""
    plan = plan_for(N, na, nd, sp, off, power_max_iter=2)
    gen = torch.Generator(device="cuda").manual_seed(3)
    for _ in range(3):
        x = torch.rand(N * N, device="cuda", generator=gen) * 2 - 1
        y = torch.rand(na * nd, device="cuda", generator=gen) * 2 - 1
        Kx = plan.apply_K(x)
        KTy = plan.apply_KT(y)
        lhs = float(torch.dot(Kx.double(), y.double()))
        rhs = float(torch.dot(x.double(), KTy.double()))
        scale = float(torch.dot(Kx.double().abs(), y.double().abs()))
        assert abs(lhs - rhs) <= 2e-6 * scale


@pytest.mark.parametrize("N,na,nd", [(4096, 6, 4100), (16, 1, 1), (12, 3, 2)])
def test_extreme_sizes_parity(N, na, nd):
    """The largest image side a plan accepts (4096: 128 x 128 gather tiles, a 4096-point FFT
    in the plan's setup), a single ray, and fewer bins than the image is wide."""
    rng = np.random.default_rng(N + 3 * na)
    x = f32(rng.uniform(-1, 1, (N, N)))
    yv = f32(rng.uniform(-1, 1, (na, nd)))
    g = oop.Geometry(N, na, nd)
    plan = plan_for(N, na, nd, power_max_iter=2)
    y = plan.apply_K(torch.from_numpy(x.ravel().astype(np.float32)).cuda())
    assert rel_l2(to_np(y), oop.K(x, g)) <= TOL
    xt = plan.apply_KT(torch.from_numpy(yv.ravel().astype(np.float32)).cuda())
    assert rel_l2(to_np(xt), oop.KT(yv, g)) <= TOL
    # the FFT solve at this side against the oracle's, with the plan's own eigenvalues
    r = f32(rng.standard_normal((N, N)))
    out = plan.apply_Minv(torch.from_numpy(r.ravel().astype(np.float32)).cuda())
    assert rel_l2(to_np(out), oci.circulant_solve(r, plan.mu().reshape(N, N))) <= TOL
    plan.close()


def test_user_angles_with_exact_ties():
    th = [0.0, 0.3, math.pi / 4, 1.1, math.pi / 2, 2.0, 3 * math.pi / 4, 3.0, math.pi - 1e-3]
    N, nd = 48, 61
    g = oop.Geometry(N, len(th), nd, theta=np.array(th))
    x = f32(np.random.default_rng(0).uniform(0, 1, (N, N)))
    yv = f32(np.random.default_rng(1).uniform(0, 1, (len(th), nd)))
    plan = plan_for(N, len(th), nd, angles=th, power_max_iter=2)
    y = plan.apply_K(torch.from_numpy(x.ravel().astype(np.float32)).cuda())
    assert rel_l2(to_np(y), oop.K(x, g)) <= TOL
    xt = plan.apply_KT(torch.from_numpy(yv.ravel().astype(np.float32)).cuda())
    assert rel_l2(to_np(xt), oop.KT(yv, g)) <= TOL


def test_angle_close_to_an_axis():
    """Rays 1/cos(1e-4) - 1 = 5e-9 pixels more than one pixel apart: the 32.32 fixed-point
    crossings still put consecutive rays at distinct positions, so K and K^T stay an exact
    pair and match the oracle."""
    th = [0.0, 1e-4, 1.0, math.pi / 2 - 1e-4]
    N, nd = 32, 46
    g = oop.Geometry(N, len(th), nd, theta=np.array(th))
    plan = plan_for(N, len(th), nd, angles=th, power_max_iter=2)
    x = f32(np.random.default_rng(3).uniform(0, 1, (N, N)))
    yv = f32(np.random.default_rng(4).uniform(0, 1, (len(th), nd)))
    y = plan.apply_K(torch.from_numpy(x.ravel().astype(np.float32)).cuda())
    assert rel_l2(to_np(y), oop.K(x, g)) <= TOL
    xt = plan.apply_KT(torch.from_numpy(yv.ravel().astype(np.float32)).cuda())
    assert rel_l2(to_np(xt), oop.KT(yv, g)) <= TOL
    plan.close()


@pytest.mark.parametrize("N", [8, 48, 96, 512])
def test_finite_differences_parity(N):
    rng = np.random.default_rng(N)
    x = f32(rng.standard_normal((N, N)))
    plan = plan_for(N, 4, 8, power_max_iter=2)
    v = plan.apply_D(torch.from_numpy(x.ravel().astype(np.float32)).cuda())
    dh, dv = oop.D(x)
    assert rel_l2(to_np(v), v_from_oracle(dh, dv)) <= 1e-7
    w = f32(rng.standard_normal(2 * N * N))
    wh, wv = v_to_oracle(w, N)
    xt = plan.apply_DT(torch.from_numpy(w.astype(np.float32)).cuda())
    assert rel_l2(to_np(xt), oop.DT(wh, wv)) <= 1e-7


@pytest.mark.parametrize("N,na,nd,tv,gamma", [(48, 60, 70, "aniso", 0.0), (96, 140, 130, "iso", 0.3),
                                               (384, 64, 386, "aniso", 0.0), (512, 720, 730, "iso", 0.0)])
def test_mu_table_rho_and_circulant_solve(N, na, nd, tv, gamma):
    """The plan's eigenvalues of M (eqs. (circ_R), (circ_D), rescaled for (A3)),
    its power-iteration rho, and the FFT solve against the oracle."""
    lam, alpha, beta = 0.01, 1.0, 3.0
    mu_ref, rho_ref = oracle_scaled_mu(N, na, nd, alpha, beta, gamma, tv)
    plan = plan_for(N, na, nd, lam=lam, alpha=alpha, beta=beta, tv=tv, gamma=gamma, power_tol=1e-9)
    _, rho = plan.power_bound()
    assert rho == pytest.approx(rho_ref, rel=1e-5)
    assert rel_l2(plan.mu(), mu_ref) <= 1e-5
    r = f32(np.random.default_rng(N).standard_normal((N, N)))
    out = plan.apply_Minv(torch.from_numpy(r.ravel().astype(np.float32)).cuda())
    assert rel_l2(to_np(out), oci.circulant_solve(r, mu_ref)) <= TOL


def test_default_power_tolerance_is_inside_the_a3_margin():
    """With the default stop (relative change 1e-6) rho = lambda_max(M^{-1} alpha A^T A) is
    within 1e-4 of the oracle's converged value (power iteration to 1e-9): the (A3) rescale's
    1e-2 margin covers it a hundred times over."""
    N, na, nd = 96, 140, 130
    _, rho_ref = oracle_scaled_mu(N, na, nd, 0.01, 0.01, 0.0, "iso")
    plan = plan_for(N, na, nd, lam=0.005, alpha=0.01, beta=0.01, tv="iso")
    _, rho = plan.power_bound()
    plan.close()
    assert rho <= rho_ref * (1 + 1e-5) and rho == pytest.approx(rho_ref, rel=1e-4)


def test_lambda_max_AtA_parity():
    N, na, nd = 64, 90, 92
    g = oop.Geometry(N, na, nd)
    P = osv.Problem(g, np.zeros((na, nd)), lam=0.01, alpha=1.0, beta=3.0)
    lm_ref, _ = osv.power_lmax_AtA(P, osv.splitmix64_uniform(0, N * N).reshape(N, N))
    plan = plan_for(N, na, nd, lam=0.01, alpha=1.0, beta=3.0)
    lm, _ = plan.power_bound()
    assert lm == pytest.approx(lm_ref, rel=1e-5)


@pytest.mark.parametrize("kind", ["ct_aniso", "ct_iso", "pet"])
def test_objective_parity(kind):
    import synth
    N, na, nd = 96, 140, 130
    g = oop.Geometry(N, na, nd)
    if kind == "pet":
        pr = synth.pet_problem(3, N, na, nd, 8, oproj(N, na, nd), total_counts=1e5)
        P = osv.Problem(g, f32(pr["b"]), lam=0.02, alpha=0.1, beta=0.1, kind="pet", kappa=1.0,
                        r_bg=f32(pr["r_bg"]))
        plan = plan_for(N, na, nd, lam=0.02, alpha=0.1, data="kl", nonneg=True, power_max_iter=2)
        x = f32(np.random.default_rng(0).uniform(-0.2, 1.0, (N, N)) * pr["x_true"].max())
        bg = torch.from_numpy(pr["r_bg"].ravel()).cuda()
    else:
        pr = synth.ct_problem(3, N, na, nd, 8, 0.01, oproj(N, na, nd))
        tv = kind.split("_")[1]
        P = osv.Problem(g, f32(pr["b"]), lam=0.3, alpha=1.0, beta=1.0, tv=tv)
        plan = plan_for(N, na, nd, lam=0.3, tv=tv, power_max_iter=2)
        x = f32(pr["x_true"] + 0.05 * np.random.default_rng(0).standard_normal((N, N)))
        bg = None
    f = plan.objective(torch.from_numpy(x.ravel().astype(np.float32)).cuda(),
                       torch.from_numpy(pr["b"].ravel()).cuda(), bg)
    assert f == pytest.approx(osv.objective(P, x), rel=1e-6)


@pytest.mark.parametrize("N,na,nd", [(64, 90, 92), (48, 60, 70)])
def test_probe_estimated_circulant_matches_oracle(N, na, nd):
    """Eq. (H-fan), least-squares form: M's projector part from SplitMix64 probe images on
    the GPU against the oracle's probe_ls of K^T K over the same (float32) images; the A3
    rescale is off (a3_margin < 0) so the raw eigenvalues are compared."""
    P, lam, alpha, beta = 4, 0.01, 0.5, 1.5
    plan = plan_for(N, na, nd, lam=lam, alpha=alpha, beta=beta, h_probes=P, a3_margin=-1.0, power_max_iter=2)
    mu_gpu = plan.mu()
    plan.close()
    g = oop.Geometry(N, na, nd)
    vs = [f32(osv.splitmix64_uniform(1 + q, N * N)).reshape(N, N) for q in range(P)]
    h = np.maximum(oci.probe_ls(lambda v: oop.KT(oop.K(v, g), g), N, vs), 0.0)
    h[0, 0] = oci.h_dc_default(g)
    mu_ref = alpha * h + (beta * beta / alpha) * oci.H_D(N)
    err = rel_l2(mu_gpu, mu_ref)
    print("H-fan mu rel L2 %.2e" % err)
    assert err <= 1e-4
