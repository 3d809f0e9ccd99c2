"""Host-side checks of the C ABI that need no GPU: the library builds and loads,
it exports every entry point include/ncs.h declares, the binding declares the
same set, and argument validation that happens before any CUDA call."""
import ctypes
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    txt = open(os.path.join(ROOT, "include", "ncs.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z_0-9]*\s*\*?\s+\**([a-z_][A-Za-z_0-9]*)\s*\(", txt, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1810_13100_gb300 import _build, binding
    _build.build()
    return binding.load_library()


def test_header_parse_sanity():
    names = header_functions()
    for must in ("ncs_plan_create", "ncs_step", "ncs_solve", "pdhg_solve", "ncs_plan_destroy"):
        assert must in names


def test_library_exports_every_header_symbol(lib):
    for name in header_functions():
        assert hasattr(lib, name), "libncs.so does not export %s" % name


def test_binding_covers_header():
    from paper_1810_13100_gb300 import binding
    assert sorted(n for n, _, _ in binding.SIGNATURES) == header_functions()


def test_options_default_and_status_strings(lib):
    from paper_1810_13100_gb300 import binding
    o = binding.default_options()
    assert math.isnan(o.beta) and math.isnan(o.h_dc) and math.isnan(o.c_r)
    assert o.a3_margin == pytest.approx(1e-2) and o.power_max_iter == 500 and o.check_every == 10
    assert o.kappa == 1.0 and o.nonneg == 0 and o.data == 0 and o.tv == 0
    assert lib.ncs_status_string(0) == b"ok"
    assert b"unsupported" in lib.ncs_status_string(-2)
    assert lib.ncs_status_string(12345) == b"unknown status"


def _create(lib, N, na=8, nd=10, lam=0.1, alpha=1.0, spacing=1.0, opt=None):
    from paper_1810_13100_gb300 import binding
    g = binding.Geometry()
    g.n_angles, g.n_det, g.det_spacing, g.det_offset = na, nd, spacing, 0.0
    h = ctypes.c_void_p()
    rc = lib.ncs_plan_create(ctypes.byref(g), N, N, lam, alpha, ctypes.byref(opt) if opt else None, ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("N,code", [(17, -2), (10, -2), (4, -1), (4098, -2), (14, -2)])
def test_plan_create_rejects_sizes_before_touching_cuda(lib, N, code):
    rc, h = _create(lib, N)
    assert rc == code and not h.value


def test_plan_create_rejects_bad_parameters(lib):
    from paper_1810_13100_gb300 import binding
    assert _create(lib, 64, alpha=0.0)[0] == -1
    assert _create(lib, 64, lam=-1.0)[0] == -1
    assert _create(lib, 64, na=0)[0] == -1
    assert _create(lib, 64, spacing=0.5)[0] == -2
    o = binding.default_options()
    o.nonneg = 1                       # nonnegativity needs the KL data term
    assert _create(lib, 64, opt=o)[0] == -1
    o = binding.default_options()
    o.power_max_iter = 0
    assert _create(lib, 64, opt=o)[0] == -1
    o = binding.default_options()
    assert o.pdhg_only == 0
    o.pdhg_only = 2
    assert _create(lib, 64, opt=o)[0] == -1
    assert lib.ncs_plan_create(None, 64, 64, 0.1, 1.0, None, None) == -1


def test_null_plan_calls_are_rejected(lib):
    assert lib.ncs_step(None, None, None, None, None, None, None, 1) == -1
    assert lib.ncs_apply_K(None, None, None) == -1
    lib.ncs_plan_destroy(None)


def _create_fan(lib, N, nv=8, nd=10, R=None, pitch=0.01, offset=0.0, views=None):
    from paper_1810_13100_gb300 import binding
    g = binding.FanGeometry()
    g.n_views, g.n_det = nv, nd
    g.src_dist = 2.0 * N if R is None else R
    g.pitch, g.offset = pitch, offset
    if views is not None:
        arr = (ctypes.c_double * len(views))(*views)
        g.views = ctypes.cast(arr, ctypes.POINTER(ctypes.c_double))
    h = ctypes.c_void_p()
    rc = lib.ncs_plan_create_fan(ctypes.byref(g), N, N, 0.1, 1.0, None, ctypes.byref(h))
    return rc, h


def test_fan_plan_create_rejects_bad_geometry_before_touching_cuda(lib):
    assert _create_fan(lib, 64, pitch=0.0)[0] == -1
    assert _create_fan(lib, 64, pitch=float("nan"))[0] == -1
    # the source must stay outside the image's circumscribed circle plus 3 pixels
    assert _create_fan(lib, 64, R=0.5 * 63 * math.sqrt(2.0) + 2.9)[0] == -1
    assert _create_fan(lib, 64, nv=2, views=[0.0, float("inf")])[0] == -1
    assert _create_fan(lib, 64, nv=0)[0] == -1
    assert _create_fan(lib, 17)[0] == -2
    assert lib.ncs_plan_create_fan(None, 64, 64, 0.1, 1.0, None, None) == -1


def test_fan_plan_rejects_unknown_gather_kernel(lib):
    from paper_1810_13100_gb300 import binding
    g = binding.FanGeometry()
    g.n_views, g.n_det, g.src_dist, g.pitch, g.offset = 8, 10, 128.0, 0.01, 0.0
    for bad in (-1, 3):
        o = binding.default_options()
        o.fan_gather = bad
        h = ctypes.c_void_p()
        assert lib.ncs_plan_create_fan(ctypes.byref(g), 64, 64, 0.1, 1.0, ctypes.byref(o), ctypes.byref(h)) == -1
        assert not h.value


def test_cone_create_rejects_bad_geometry_before_touching_cuda(lib):
    from paper_1810_13100_gb300 import binding

    def create(N=16, Nz=4, nv=4, nr=5, nd=8, R=20.0, pitch=0.05, rp=0.1, roff=0.0):
        g = binding.ConeGeometry()
        g.n_views, g.n_rows, g.n_det = nv, nr, nd
        g.src_dist, g.pitch, g.offset, g.row_pitch, g.row_offset = R, pitch, 0.0, rp, roff
        h = ctypes.c_void_p()
        rc = lib.ncs_cone_create(ctypes.byref(g), N, Nz, None, ctypes.byref(h))
        assert not h.value
        return rc
    assert create(rp=0.4) == -1            # outer slopes +-0.8 >= 1/sqrt(2)
    assert create(roff=0.7) == -1
    assert create(R=12.0) == -1            # source inside the image's circle plus 3 pixels
    assert create(pitch=0.0) == -1 and create(rp=-0.1) == -1
    assert create(N=15) == -1 and create(Nz=0) == -1 and create(nr=0) == -1
    assert lib.ncs_cone_create(None, 16, 4, None, None) == -1
