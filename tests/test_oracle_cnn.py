"""Pins of the U-Net oracle: the convolution against its definition as a direct
sum, the data and weight gradients as adjoints (<conv(x), g> identities), the
pooling / upsampling adjoint pair, and the full gradient against central finite
differences in FP64."""
import numpy as np
import pytest

from oracle import cnn


def test_conv_matches_direct_sum():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((5, 6, 3))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    out = cnn.conv3x3(x, w, b)
    ref = np.zeros((5, 6, 4))
    for y in range(5):
        for xx in range(6):
            for co in range(4):
                s = b[co]
                for kh in range(3):
                    for kw in range(3):
                        yy, xs = y + kh - 1, xx + kw - 1
                        if 0 <= yy < 5 and 0 <= xs < 6:
                            s += np.dot(x[yy, xs], w[co, kh, kw])
                ref[y, xx, co] = s
    assert np.allclose(out, ref, atol=1e-12)


def test_conv_gradients_are_adjoints():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((6, 4, 3))
    w = rng.standard_normal((5, 3, 3, 3))
    g = rng.standard_normal((6, 4, 5))
    lhs = np.sum(cnn.conv3x3(x, w) * g)
    assert np.sum(x * cnn.conv3x3_dgrad(g, w)) == pytest.approx(lhs, rel=1e-12)
    assert np.sum(w * cnn.conv3x3_wgrad(g, x)) == pytest.approx(lhs, rel=1e-12)


def test_pool_up_adjoints():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((8, 6, 3))
    g = rng.standard_normal((4, 3, 3))
    assert np.sum(cnn.pool(x) * g) == pytest.approx(np.sum(x * cnn.pool_bwd(g)), rel=1e-12)
    z = rng.standard_normal((4, 3, 3))
    h = rng.standard_normal((8, 6, 3))
    assert np.sum(cnn.up(z) * h) == pytest.approx(np.sum(z * cnn.up_bwd(h)), rel=1e-12)


def test_bf16_rounding():
    # bfloat16 keeps 8 significant bits: its ulp at 1 is 2^-7
    assert cnn.bf16(1.0) == 1.0
    assert cnn.bf16(1.0 + 2.0 ** -9) == 1.0                   # a quarter ulp: down
    assert cnn.bf16(1.0 + 3 * 2.0 ** -9) == 1.0 + 2.0 ** -7   # three quarters of an ulp: up
    assert cnn.bf16(1.0 + 2.0 ** -8) == 1.0                   # a tie: to the even neighbour, down
    assert cnn.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6   # a tie: to the even neighbour, up
    assert cnn.bf16(-(1.0 + 2.0 ** -8)) == -1.0               # ties to even on the negative side too


@pytest.mark.parametrize("levels,base,H", [(2, 2, 8), (3, 2, 8)])
def test_gradient_matches_finite_differences(levels, base, H):
    rng = np.random.default_rng(3)
    n = cnn.n_params(levels, base)
    p = rng.standard_normal(n) * 0.5
    x = rng.standard_normal((H, H))
    t = rng.standard_normal((H, H))
    net = cnn.UNetOracle(levels, base, emulate=False)
    loss, g, _ = net.loss_and_grad(p, x, t)
    for trial in range(3):
        d = rng.standard_normal(n)
        eps = 1e-6
        lp, _, _ = net.loss_and_grad(p + eps * d, x, t)
        lm, _, _ = net.loss_and_grad(p - eps * d, x, t)
        fd = (lp - lm) / (2 * eps)
        assert fd == pytest.approx(np.dot(g, d), rel=1e-5, abs=1e-9)
    # a few single coordinates, including the head and the first convolution
    for i in (0, n // 3, n - 2, n - 1):
        e = np.zeros(n)
        e[i] = 1.0
        lp, _, _ = net.loss_and_grad(p + 1e-6 * e, x, t)
        lm, _, _ = net.loss_and_grad(p - 1e-6 * e, x, t)
        assert (lp - lm) / 2e-6 == pytest.approx(g[i], rel=1e-4, abs=1e-8)
