"""GPU parity of the warm-start parts (not in the paper) against the FP64 oracle:
the Ram-Lak filtered backprojection, the consistent dual start u^0 = K x^0 - b,
and the U-Net's forward output and parameter gradient (the oracle emulates the
GPU's bfloat16 rounding points, so the remaining differences are FP32 versus
FP64 accumulation and rare one-ulp bfloat16 rounding flips)."""
import numpy as np
import pytest

import synth
from helpers import f32, oproj, oracle_scaled_mu, rel_l2, to_np
from oracle import cnn as ocnn
from oracle import fbp as ofbp
from oracle import operators as oop
from oracle import solvers as osv

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N,na,nd,sp", [(96, 140, 130, 1.0), (512, 720, 730, 1.0), (64, 50, 61, 1.5)])
def test_fbp_parity(N, na, nd, sp):
    import paper_1810_13100_gb300 as ncs
    pr = synth.ct_problem(2, N, na, nd, 8, 0.01, oproj(N, na, nd, spacing=sp), det_spacing=sp)
    g = oop.Geometry(N, na, nd, spacing=sp)
    plan = ncs.Plan(N, na, nd, 0.01, 1.0, det_spacing=sp, power_max_iter=2)
    x = plan.fbp(torch.from_numpy(pr["b"].ravel()).cuda())
    ref = ofbp.fbp(f32(pr["b"]), g)
    assert rel_l2(to_np(x), ref) <= 2e-5
    plan.close()


def test_warm_dual_start_parity():
    """From x^0 (a seeded image) with u^0 = K x^0 - b, 10 NCS iterations on the GPU
    match the oracle's iterations from the same start."""
    import paper_1810_13100_gb300 as ncs
    N, na, nd = 96, 140, 130
    lam, alpha, beta = 0.3, 1.0, 3.0
    pr = synth.ct_problem(3, N, na, nd, 8, 0.01, oproj(N, na, nd))
    g = oop.Geometry(N, na, nd)
    P = osv.Problem(g, f32(pr["b"]), lam=lam, alpha=alpha, beta=beta, tv="iso")
    x0 = f32(pr["x_true"] + 0.05 * np.random.default_rng(0).standard_normal((N, N)))
    plan = ncs.Plan(N, na, nd, lam, alpha, beta=beta, tv="iso", warm_dual=True, power_tol=1e-9)
    x = torch.from_numpy(x0.ravel().astype(np.float32)).cuda()
    plan.solve(torch.from_numpy(pr["b"].ravel()).cuda(), x, tol=0.0, max_iter=10, f_star=-1e300)
    mus, _ = oracle_scaled_mu(N, na, nd, alpha, beta, 0.0, "iso")
    st = osv.zero_state(P)
    st.x = x0.copy()
    st.u = oop.K(x0, g) - P.b
    st = osv.run(P, st, 10, osv.circulant_Minv(mus))
    assert rel_l2(to_np(x), st.x) <= 2e-4
    plan.close()


def rand_params(levels, base, seed):
    rng = np.random.default_rng(seed)
    convs, c = ocnn.layout(levels, base)
    parts = []
    for cin, cout in convs:
        parts.append(rng.standard_normal(cout * 9 * cin) * np.sqrt(2.0 / (9 * cin)))
        parts.append(rng.uniform(-0.05, 0.05, cout))
    parts.append(rng.standard_normal(c[0]) * 0.1)
    parts.append(np.array([0.01]))
    return np.concatenate(parts).astype(np.float32)


def smooth_image(H, seed):
    rng = np.random.default_rng(seed)
    yy, xx = np.meshgrid(np.linspace(-1, 1, H), np.linspace(-1, 1, H), indexing="ij")
    img = np.zeros((H, H))
    for _ in range(5):
        cx, cy, r, v = rng.uniform(-0.6, 0.6), rng.uniform(-0.6, 0.6), rng.uniform(0.1, 0.5), rng.uniform(0.2, 1)
        img += v * (((xx - cx) ** 2 + (yy - cy) ** 2) < r * r)
    return (img + 0.05 * rng.standard_normal((H, H))).astype(np.float32)


@pytest.mark.parametrize("levels,base,H", [(3, 8, 32), (4, 8, 64), (2, 32, 32), (2, 160, 8)])
def test_unet_forward_and_gradient_parity(levels, base, H):
    import paper_1810_13100_gb300 as ncs
    net = ncs.UNet(H, H, levels=levels, base=base, seed=1)
    assert net.n_params == ocnn.n_params(levels, base)
    p = rand_params(levels, base, 7)
    net.set_params(p)
    x = smooth_image(H, 1)
    t = smooth_image(H, 2)
    xg = torch.from_numpy(x.ravel()).cuda()
    tg = torch.from_numpy(t.ravel()).cuda()
    y = to_np(net.forward(xg)).reshape(H, H)
    loss, grad = net.gradient(xg, tg)
    oracle = ocnn.UNetOracle(levels, base, emulate=True)
    loss_ref, grad_ref, y_ref = oracle.loss_and_grad(p.astype(np.float64), x.astype(np.float64), t.astype(np.float64))
    out_err = rel_l2(y - x, y_ref - x)
    grad_err = rel_l2(grad, grad_ref)
    print("levels %d base %d H %d: output rel L2 %.2e, gradient rel L2 %.2e, loss %.6e vs %.6e"
          % (levels, base, H, out_err, grad_err, loss, loss_ref))
    assert out_err <= 1e-2
    assert loss == pytest.approx(loss_ref, rel=1e-3)
    assert grad_err <= 3e-2
    # every convolution's weight gradient separately
    convs, c = ocnn.layout(levels, base)
    off = 0
    for cin, cout in convs:
        nw = cout * 9 * cin
        assert rel_l2(grad[off:off + nw], grad_ref[off:off + nw]) <= 6e-2
        off += nw + cout
    net.close()


def test_unet_training_decreases_loss():
    import paper_1810_13100_gb300 as ncs
    H = 64
    net = ncs.UNet(H, H, levels=4, base=8, seed=3)
    x = torch.from_numpy(smooth_image(H, 5).ravel()).cuda()
    t = torch.from_numpy((smooth_image(H, 5) * 0.8 + 0.1).ravel()).cuda()
    losses = [net.train_step(x, t, 1e-3) for _ in range(60)]
    assert losses[-1] < 0.5 * losses[0], losses[::10]
    net.close()


def test_learned_start_needs_fewer_iterations_than_fbp_and_zero():
    """The warm-start pipeline end to end at 128x128 (180 angles, 130 bins, iso TV
    lambda 1, alpha = beta = 0.3, where TV is active): 64 training pairs made by
    plain NCS on the GPU, a 3-level U-Net trained on them with the library's
    kernels, then 8 fresh seeds.  Plain NCS from the learned x^0 reaches the 1e-4
    gap (against plain NCS from zero after 5000 iterations) in fewer iterations
    than from FBP or zero; the held-out error of the network falls."""
    import paper_1810_13100_gb300 as ncs
    from paper_1810_13100_gb300 import warmstart as wsm
    N, na, nd, lam, al = 128, 180, 130, 1.0, 0.3
    proj = oproj(N, na, nd)

    def sinos(seeds):
        for s in seeds:
            yield torch.from_numpy(synth.ct_problem(s, N, na, nd, 20, 0.005, proj)["b"].ravel()).cuda()

    plans = [ncs.Plan(N, na, nd, lam, al, beta=al, tv="iso") for _ in range(2)]
    ins, outs = wsm.make_pairs(plans, sinos(range(100, 164)), 1000)
    ws = wsm.WarmStart(plans[0], 3, 16, seed=1)
    hist = wsm.train(ws, ins, outs, 30, lr=1e-3)
    assert hist[-1]["val_mse"] < 0.5 * hist[0]["val_mse"], [h["val_mse"] for h in hist]
    res = wsm.evaluate(plans, ws, list(sinos(range(900, 908))), tol=1e-4, cap=3000, ref_iters=5000)
    mean = {nm: np.mean([r[nm]["iters"] for r in res]) for nm in ("zero", "fbp", "learned")}
    print("mean iterations to 1e-4:", mean)
    assert all(r[nm]["iters"] is not None for r in res for nm in mean)
    assert mean["learned"] <= 0.95 * mean["fbp"]
    assert mean["learned"] < mean["zero"]
    # the learned x^0 is closer to the minimiser in objective than FBP on every seed
    assert all(r["learned"]["gap0"] < r["fbp"]["gap0"] for r in res)
    ws.close()
    for p in plans:
        p.close()


def test_unet_tensor_core_path_matches_mma_sync_path():
    """The tcgen05 convolutions (tensor-memory accumulators) against the mma.sync ones on
    the 4-level, base-32 512x512 network: same forward output and gradient up to FP32
    accumulation order (both round the same bf16 operands)."""
    import paper_1810_13100_gb300 as ncs
    H = 512
    x = torch.from_numpy(smooth_image(H, 3).ravel()).cuda()
    t = torch.from_numpy(smooth_image(H, 4).ravel()).cuda()
    net = ncs.UNet(H, H, levels=4, base=32, seed=5)
    p = rand_params(4, 32, 11)
    net.set_params(p)
    net.set_conv_path(False)
    y0 = to_np(net.forward(x))
    l0, g0 = net.gradient(x, t)
    net.set_conv_path(True)
    y1 = to_np(net.forward(x))
    l1, g1 = net.gradient(x, t)
    xin = to_np(x)
    print("tc vs mma.sync: output %.2e, gradient %.2e" % (rel_l2(y1 - xin, y0 - xin), rel_l2(g1, g0)))
    assert rel_l2(y1 - xin, y0 - xin) <= 5e-3
    assert l1 == pytest.approx(l0, rel=1e-3)
    assert rel_l2(g1, g0) <= 2e-2
    net.close()
