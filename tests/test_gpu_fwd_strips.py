"""The strip form of the parallel-beam K (image rows staged in shared memory, one pass per
strip and a fixed-order sum of the strips) against the FP64 oracle and against the row walk
(each ray reads its rows from L2): both evaluate the same 32.32 crossings and weights and
differ only in the FP32 summation order.

Cases: strip counts 1 to 14 with ragged last strips (N = 512: 5 strips of 103 rows with 100
in the last; N = 864: 14 of 62 with 58 in the last), bin counts that leave a partial warp, angle sets with
an empty branch (every angle within 30 degrees of the x axis, or of the y axis), a single
ray, and every epilogue of the forward pass inside NCS iterations (L2 data prox with the
running K x and its FP64 data term, the KL prox, both objective sums), with FP32 and with
bfloat16 pair images.  Tolerance: 1e-5 relative L2 against the oracle (the FP32 operator
bound of the other tests); strips against the row walk: 1e-6 per operator (the order of
<= 2N FP32 additions), 1e-5 after 20 iterations."""
import math

import numpy as np
import pytest

import synth
from helpers import f32, oproj, rel_l2, to_np
from oracle import operators as oop

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def plan(N, na, nd, kernel, **kw):
    import paper_1810_13100_gb300 as ncs
    kw.setdefault("power_max_iter", 2)
    lam = kw.pop("lam", 0.01)
    alpha = kw.pop("alpha", 1.0)
    return ncs.Plan(N, na, nd, lam, alpha, fwd_kernel=kernel, **kw)


@pytest.mark.parametrize("N,na,nd,strips", [(32, 48, 46, 1), (96, 140, 130, 1), (256, 90, 258, 2),
                                            (384, 64, 386, 3), (512, 720, 730, 5), (648, 40, 650, 8),
                                            (864, 24, 866, 14)])
def test_strip_forward_against_oracle_and_row_walk(N, na, nd, strips):
    rng = np.random.default_rng(N + nd)
    x = f32(rng.uniform(-1, 1, (N, N)))
    ref = oop.K(x, oop.Geometry(N, na, nd))
    xt = torch.from_numpy(x.ravel().astype(np.float32)).cuda()
    ps, pr = plan(N, na, nd, "strips"), plan(N, na, nd, "rows")
    assert ps.fwd_strips()[0] == strips and pr.fwd_strips() == (0, 0)
    ys, yr = to_np(ps.apply_K(xt)), to_np(pr.apply_K(xt))
    assert rel_l2(ys, ref) <= TOL and rel_l2(yr, ref) <= TOL
    assert rel_l2(ys, yr) <= 1e-6
    ps.close()
    pr.close()


@pytest.mark.parametrize("theta", [
    [0.0, 0.1, 0.25, -0.3 + math.pi, 0.5],                       # row branch only
    [math.pi / 2, 1.2, 1.9, math.pi / 2 + 0.4],                   # column branch only
    [0.0, 1e-4, math.pi / 4, math.pi / 2 - 1e-4, 3 * math.pi / 4],  # ties and near-axis angles
])
def test_strip_forward_with_an_empty_branch(theta):
    N, nd = 384, 37                                               # 3 strips; 37 bins: one partial warp
    g = oop.Geometry(N, len(theta), nd, theta=np.array(theta))
    x = f32(np.random.default_rng(5).uniform(0, 1, (N, N)))
    p = plan(N, len(theta), nd, "strips", angles=theta)
    assert p.fwd_strips()[0] == 3
    y = p.apply_K(torch.from_numpy(x.ravel().astype(np.float32)).cuda())
    assert rel_l2(to_np(y), oop.K(x, g)) <= TOL
    p.close()


def test_strip_forward_single_ray_and_bf16_pairs():
    import paper_1810_13100_gb300 as ncs
    N = 256
    x = f32(np.random.default_rng(9).uniform(-1, 1, (N, N)))
    xt = torch.from_numpy(x.ravel().astype(np.float32)).cuda()
    p1 = plan(N, 1, 1, "strips")
    assert rel_l2(to_np(p1.apply_K(xt)), oop.K(x, oop.Geometry(N, 1, 1))) <= TOL
    p1.close()
    # bfloat16 pair images: both kernels read the same rounded values
    na, nd = 180, 258
    ps, pr = plan(N, na, nd, "strips"), plan(N, na, nd, "rows")
    assert rel_l2(to_np(ps.apply_K_bf16(xt)), to_np(pr.apply_K_bf16(xt))) <= 1e-6
    ps.close()
    pr.close()


@pytest.mark.parametrize("kind", ["ct", "pet"])
def test_strip_forward_inside_iterations(kind):
    """20 NCS iterations with each K kernel from the same zero state: the prox epilogues (L2
    with the running K x in a solve, KL), the FP64 objective sums and the strip sum agree."""
    N, na, nd = 256, 180, 258
    if kind == "ct":
        pr_ = synth.ct_problem(2, N, na, nd, 10, 0.01, oproj(N, na, nd))
        kw = dict(lam=0.01, alpha=0.1, tv="iso", power_tol=1e-9)
        bg = None
    else:
        pr_ = synth.pet_problem(2, N, na, nd, 10, oproj(N, na, nd), total_counts=1e6)
        kw = dict(lam=0.02, alpha=0.1, tv="aniso", data="kl", nonneg=True, power_tol=1e-9)
        bg = torch.from_numpy(pr_["r_bg"].ravel().astype(np.float32)).cuda()
    b = torch.from_numpy(pr_["b"].ravel().astype(np.float32)).cuda()
    out = {}
    for kernel in ("strips", "rows"):
        p = plan(N, na, nd, kernel, **dict(kw))
        x = torch.zeros(N * N, device="cuda")
        if kind == "ct":
            rep = p.solve(b, x, tol=0.0, max_iter=20, f_star=-1e300)
            f = rep["f"]
        else:
            u = torch.zeros(na * nd, device="cuda")
            v = torch.zeros(2 * N * N, device="cuda")
            s = torch.zeros(N * N, device="cuda")
            p.step(x, u, v, s, b, bg, n_iter=20)
            f = p.objective(x, b, bg)
        out[kernel] = (to_np(x), f)
        p.close()
    assert rel_l2(out["strips"][0], out["rows"][0]) <= 1e-5
    assert abs(out["strips"][1] - out["rows"][1]) <= 1e-6 * abs(out["rows"][1])


def test_strip_option_errors():
    import paper_1810_13100_gb300 as ncs
    from paper_1810_13100_gb300 import binding
    # 1024 x 1024 has no strip pitch: "strips" is refused, "auto" takes the row walk
    with pytest.raises(binding.NCSError) as e:
        plan(1024, 4, 1026, "strips", pdhg_only=True)
    assert e.value.code == binding.NCS_ERR_UNSUPPORTED
    p = plan(1024, 4, 1026, "auto", pdhg_only=True)
    assert p.fwd_strips() == (0, 0)
    p.close()
    # the fan beam has no strip form
    pf = ncs.Plan(64, 60, 70, 0.01, 1.0, src_dist=128.0, fan_pitch=0.012, power_max_iter=2, pdhg_only=True)
    assert pf.fwd_strips() == (0, 0)
    pf.close()
