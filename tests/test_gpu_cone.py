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
