"""ncs_apply_KT_static: the backprojection for callers that cannot allocate
device memory (it takes its working memory from a static device array instead
of a plan).  Checked through the C ABI against the plan-based ncs_apply_KT on
two calls in a row, and against the FP64 oracle's K^T, within the operator
tolerance of the other tests, and for its size limits and status codes.  Kept in
its own file, collected last."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


def _geom(binding, na, nd):
    g = binding.Geometry()
    g.n_angles, g.n_det, g.det_spacing, g.det_offset = na, nd, 1.0, 0.0
    g.angles = None
    return g


@pytest.mark.parametrize("N,na,nd", [(512, 720, 730), (96, 140, 130)])
def test_static_backprojection_matches_plan_on_two_calls(N, na, nd):
    import paper_1810_13100_gb300 as ncs
    from paper_1810_13100_gb300 import binding
    from oracle import operators as oop
    L = binding.load_library()
    plan = ncs.Plan(N, na, nd, 0.01, 1.0, power_max_iter=2)
    g = _geom(binding, na, nd)
    og = oop.Geometry(N, na, nd)
    gen = torch.Generator(device="cuda").manual_seed(11)
    for call in range(2):
        y = torch.rand(na * nd, device="cuda", generator=gen) * 2 - 1
        ref = plan.apply_KT(y)
        out = torch.full((N * N,), float("nan"), device="cuda")
        torch.cuda.synchronize()
        rc = L.ncs_apply_KT_static(ctypes.byref(g), N, ctypes.c_void_p(y.data_ptr()),
                                   ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(0))
        assert rc == 0, binding.status_string(rc)
        torch.cuda.synchronize()
        a = out.double().cpu().numpy()
        r = ref.double().cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - r) <= TOL * np.linalg.norm(r), call
        # the same product from the FP64 oracle on the same float32 sinogram
        o = oop.KT(y.double().cpu().numpy().reshape(na, nd), og).ravel()
        assert np.linalg.norm(a - o) <= TOL * np.linalg.norm(o), call
    plan.close()


def test_static_backprojection_rejects_sizes_beyond_its_limit():
    from paper_1810_13100_gb300 import binding
    L = binding.load_library()
    g = _geom(binding, 8, 10)
    dummy = torch.zeros(1, device="cuda")
    p = ctypes.c_void_p(dummy.data_ptr())
    assert L.ncs_apply_KT_static(ctypes.byref(g), 768, p, p, None) == binding.NCS_ERR_UNSUPPORTED
    g2 = _geom(binding, 4096, 10)
    assert L.ncs_apply_KT_static(ctypes.byref(g2), 64, p, p, None) == binding.NCS_ERR_UNSUPPORTED
    assert L.ncs_apply_KT_static(ctypes.byref(g), 4, p, p, None) == binding.NCS_ERR_BADARG
    g3 = _geom(binding, 8, 10)
    g3.det_spacing = 0.5
    assert L.ncs_apply_KT_static(ctypes.byref(g3), 64, p, p, None) == binding.NCS_ERR_UNSUPPORTED
    assert L.ncs_apply_KT_static(None, 64, p, p, None) == binding.NCS_ERR_BADARG


def test_static_backprojection_refuses_graph_capture():
    """On a stream that is capturing a CUDA graph the call returns NCS_ERR_UNSUPPORTED and
    enqueues nothing (its angle table is copied from host memory the call owns); the same
    call outside the capture succeeds."""
    from paper_1810_13100_gb300 import binding
    L = binding.load_library()
    N, na, nd = 64, 90, 92
    g = _geom(binding, na, nd)
    y = torch.rand(na * nd, device="cuda")
    out = torch.zeros(N * N, device="cuda")
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        rc = L.ncs_apply_KT_static(ctypes.byref(g), N, ctypes.c_void_p(y.data_ptr()),
                                   ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(s.cuda_stream))
        out.add_(0.0)    # one captured torch op, so the graph is not empty
    assert rc == binding.NCS_ERR_UNSUPPORTED
    rc = L.ncs_apply_KT_static(ctypes.byref(g), N, ctypes.c_void_p(y.data_ptr()),
                               ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(s.cuda_stream))
    s.synchronize()
    assert rc == 0 and torch.isfinite(out).all()
