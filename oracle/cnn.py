"""FP64 oracle for the warm-start U-Net (not in the paper).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Plain numpy: NHWC tensors, 3x3 cross-correlation with zero padding (tap (kh, kw)
reads pixel (y + kh - 1, x + kw - 1)), ReLU, 2x2 average pooling, nearest 2x
upsampling, channel concatenation [upsampled | skip], a 1x1 head, y = x + net(x),
loss mean((y - t)^2), and the gradient by the chain rule written out layer by
layer.  With emulate=True the values are rounded to bfloat16 (round to nearest
even) at the points where the GPU stores bfloat16: the input image, the weights
used by the convolutions, every activation, the pooled maps and the masked
gradients that enter the tensor-core products; everything else stays FP64.

Parameter order (as in include/ncs.h): per convolution in creation order
(encoder levels top down, two each; decoder levels bottom up, two each) weights
[Cout][3][3][Cin] then biases [Cout]; then the head weights [base] and bias [1].
"""
from __future__ import annotations

import numpy as np


def bf16(a):
    """Round to bfloat16 (round to nearest even) and return float64."""
    a32 = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = a32.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def conv3x3(x, w, b=None):
    """x: (H, W, Cin), w: (Cout, 3, 3, Cin) -> (H, W, Cout)."""
    H, W, _ = x.shape
    xp = np.pad(x, ((1, 1), (1, 1), (0, 0)))
    out = np.zeros((H, W, w.shape[0]))
    for kh in range(3):
        for kw in range(3):
            out += xp[kh:kh + H, kw:kw + W, :] @ w[:, kh, kw, :].T
    if b is not None:
        out += b
    return out


def conv3x3_wgrad(g, x):
    """dW[co, kh, kw, ci] = sum_p g[p, co] x[p + (kh-1, kw-1), ci]."""
    H, W, Cout = g.shape
    xp = np.pad(x, ((1, 1), (1, 1), (0, 0)))
    dw = np.zeros((Cout, 3, 3, x.shape[2]))
    for kh in range(3):
        for kw in range(3):
            dw[:, kh, kw, :] = g.reshape(-1, Cout).T @ xp[kh:kh + H, kw:kw + W, :].reshape(-1, x.shape[2])
    return dw


def conv3x3_dgrad(g, w):
    """Adjoint of conv3x3 in x: correlation with the flipped, transposed kernel."""
    wf = w[:, ::-1, ::-1, :].transpose(3, 1, 2, 0)      # (Cin, 3, 3, Cout)
    return conv3x3(g, wf)


def pool(x):
    H, W, C = x.shape
    return 0.25 * x.reshape(H // 2, 2, W // 2, 2, C).sum(axis=(1, 3))


def pool_bwd(g):
    return 0.25 * np.repeat(np.repeat(g, 2, axis=0), 2, axis=1)


def up(x):
    return np.repeat(np.repeat(x, 2, axis=0), 2, axis=1)


def up_bwd(g):
    H, W, C = g.shape
    return g.reshape(H // 2, 2, W // 2, 2, C).sum(axis=(1, 3))


def layout(levels, base):
    """List of (cin, cout) per convolution in parameter order, and the head size."""
    c = [base << l for l in range(levels)]
    convs = []
    for l in range(levels):
        convs.append((1 if l == 0 else c[l - 1], c[l]))
        convs.append((c[l], c[l]))
    for l in range(levels - 2, -1, -1):
        convs.append((c[l + 1] + c[l], c[l]))
        convs.append((c[l], c[l]))
    return convs, c


def unpack(params, levels, base):
    convs, c = layout(levels, base)
    out, off = [], 0
    for cin, cout in convs:
        n = cout * 9 * cin
        w = params[off:off + n].reshape(cout, 3, 3, cin)
        off += n
        b = params[off:off + cout]
        off += cout
        out.append((w, b))
    hw = params[off:off + c[0]]
    hb = params[off + c[0]]
    assert off + c[0] + 1 == params.size
    return out, hw, hb


def n_params(levels, base):
    convs, c = layout(levels, base)
    return sum(co * 9 * ci + co for ci, co in convs) + c[0] + 1


class UNetOracle:
    """Forward and backward of the U-Net in float64 (optionally emulating bf16)."""

    def __init__(self, levels, base, emulate=False):
        self.levels, self.base, self.emulate = levels, base, emulate

    def _r(self, a):
        return bf16(a) if self.emulate else a

    def loss_and_grad(self, params, x, t):
        """x, t: (H, W) images; returns (loss, gradient in parameter order, y)."""
        L = self.levels
        r = self._r
        params = np.asarray(params, dtype=np.float64)
        layers, hw, hb = unpack(params, L, self.base)
        wq = [r(w) for w, _ in layers]
        convs, c = layout(L, self.base)
        H, W = x.shape
        idx = {}
        k = 0
        for l in range(L):
            idx[("ea", l)] = k
            idx[("eb", l)] = k + 1
            k += 2
        for l in range(L - 2, -1, -1):
            idx[("da", l)] = k
            idx[("db", l)] = k + 1
            k += 2
        relu = lambda z: np.maximum(z, 0.0)
        # ---------------- forward
        inp = {0: r(np.asarray(x, dtype=np.float64)[:, :, None])}
        act_a, skip, outl, cat, d1 = {}, {}, {}, {}, {}
        for l in range(L):
            ia = idx[("ea", l)]
            act_a[l] = r(relu(conv3x3(inp[l], wq[ia], layers[ia][1])))
            ib = idx[("eb", l)]
            e = r(relu(conv3x3(act_a[l], wq[ib], layers[ib][1])))
            if l < L - 1:
                skip[l] = e
                inp[l + 1] = r(pool(e))
            else:
                outl[l] = e
        for l in range(L - 2, -1, -1):
            cat[l] = np.concatenate([up(outl[l + 1]), skip[l]], axis=2)
            ia = idx[("da", l)]
            d1[l] = r(relu(conv3x3(cat[l], wq[ia], layers[ia][1])))
            ib = idx[("db", l)]
            outl[l] = r(relu(conv3x3(d1[l], wq[ib], layers[ib][1])))
        h = outl[0]
        y = np.asarray(x, dtype=np.float64) + h @ hw + hb
        diff = y - t
        loss = float(np.mean(diff * diff))
        # ---------------- backward
        grads = [None] * len(layers)
        dy = 2.0 * diff / diff.size
        g_h = dy[:, :, None] * hw[None, None, :]
        g_hw = np.einsum("ij,ijc->c", dy, h)
        g_hb = dy.sum()

        def conv_bwd(i, g_out, y_out, x_in, need_in=True):
            gm = r(g_out * (y_out > 0))
            grads[i] = (conv3x3_wgrad(gm, x_in), gm.sum(axis=(0, 1)))
            return conv3x3_dgrad(gm, wq[i]) if need_in else None

        g_out = {0: g_h}
        g_cat = {}
        for l in range(0, L - 1):
            g_d1 = conv_bwd(idx[("db", l)], g_out[l], outl[l], d1[l])
            g_cat[l] = conv_bwd(idx[("da", l)], g_d1, d1[l], cat[l])
            cn = c[l + 1]
            g_out[l + 1] = up_bwd(g_cat[l][:, :, :cn])
        g_in = {}
        for l in range(L - 1, -1, -1):
            if l == L - 1:
                g_e, e_out = g_out[l], outl[l]
            else:
                cn = c[l + 1]
                g_e = pool_bwd(g_in[l + 1]) + g_cat[l][:, :, cn:]
                e_out = skip[l]
            g_a = conv_bwd(idx[("eb", l)], g_e, e_out, act_a[l])
            g_in[l] = conv_bwd(idx[("ea", l)], g_a, act_a[l], inp[l], need_in=l > 0)
        flat = []
        for dw, db in grads:
            flat.append(dw.ravel())
            flat.append(db.ravel())
        flat.append(g_hw.ravel())
        flat.append(np.array([g_hb]))
        return loss, np.concatenate(flat), y
