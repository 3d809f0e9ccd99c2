"""ctypes binding of the C ABI in include/ncs.h (argument marshalling only).

Every numerical step runs in libncs.so; this module only converts torch CUDA
tensors to device pointers, fills the C structs and maps status codes to
exceptions.  There is no CPU fallback: if the library is missing the import of
the plan class fails with a clear error.
"""
from __future__ import annotations

import ctypes
import math
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libncs.so")

NCS_OK = 0
NCS_NOT_CONVERGED = 1
NCS_ERR_BADARG = -1
NCS_ERR_UNSUPPORTED = -2
NCS_ERR_CUDA = -3
NCS_ERR_NOMEM = -4
NCS_ERR_DIVERGED = -5
NCS_ERR_TIMEOUT = -6


class NCSError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        super().__init__("%s: %s (status %d)" % (what, status_string(code), code))


class Geometry(ctypes.Structure):
    _fields_ = [("n_angles", ctypes.c_int), ("n_det", ctypes.c_int),
                ("det_spacing", ctypes.c_double), ("det_offset", ctypes.c_double),
                ("angles", ctypes.POINTER(ctypes.c_double))]


class FanGeometry(ctypes.Structure):
    _fields_ = [("n_views", ctypes.c_int), ("n_det", ctypes.c_int), ("src_dist", ctypes.c_double),
                ("pitch", ctypes.c_double), ("offset", ctypes.c_double),
                ("views", ctypes.POINTER(ctypes.c_double))]


class ConeGeometry(ctypes.Structure):
    _fields_ = [("n_views", ctypes.c_int), ("n_rows", ctypes.c_int), ("n_det", ctypes.c_int),
                ("src_dist", ctypes.c_double), ("pitch", ctypes.c_double), ("offset", ctypes.c_double),
                ("row_pitch", ctypes.c_double), ("row_offset", ctypes.c_double),
                ("views", ctypes.POINTER(ctypes.c_double))]


class Options(ctypes.Structure):
    _fields_ = [("beta", ctypes.c_double), ("gamma", ctypes.c_double), ("h_dc", ctypes.c_double),
                ("c_r", ctypes.c_double), ("kappa", ctypes.c_double),
                ("data", ctypes.c_int), ("tv", ctypes.c_int), ("nonneg", ctypes.c_int), ("prec", ctypes.c_int),
                ("a3_margin", ctypes.c_double), ("power_max_iter", ctypes.c_int), ("power_tol", ctypes.c_double),
                ("power_seed", ctypes.c_uint64), ("check_every", ctypes.c_int), ("cuda_stream", ctypes.c_void_p),
                ("autotune", ctypes.c_int), ("warm_dual", ctypes.c_int), ("h_probes", ctypes.c_int),
                ("fan_gather", ctypes.c_int), ("pdhg_only", ctypes.c_int), ("fwd_kernel", ctypes.c_int)]


class Report(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("status", ctypes.c_int), ("time_ms", ctypes.c_double),
                ("f", ctypes.c_double), ("gap", ctypes.c_double), ("rho", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None

# (name, restype, argtypes) of every exported entry point
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)
SIGNATURES = [
    ("ncs_options_default", None, [ctypes.POINTER(Options)]),
    ("ncs_plan_create", _I, [ctypes.POINTER(Geometry), _I, _I, _D, _D, ctypes.POINTER(Options), ctypes.POINTER(_P)]),
    ("ncs_plan_create_fan", _I, [ctypes.POINTER(FanGeometry), _I, _I, _D, _D, ctypes.POINTER(Options),
                                 ctypes.POINTER(_P)]),
    ("ncs_plan_destroy", None, [_P]),
    ("ncs_step", _I, [_P, _P, _P, _P, _P, _P, _P, _I]),
    ("pdhg_step", _I, [_P, _P, _P, _P, _P, _P, _P, _I]),
    ("ncs_solve", _I, [_P, _P, _P, _P, _D, _I, _D, ctypes.POINTER(Report)]),
    ("pdhg_solve", _I, [_P, _P, _P, _P, _D, _I, _D, ctypes.POINTER(Report)]),
    ("admm_solve", _I, [_P, _P, _P, _D, _I, _I, _D, ctypes.POINTER(Report)]),
    ("ncs_power_bound", _I, [_P, _DP, _DP]),
    ("ncs_apply_K", _I, [_P, _P, _P]),
    ("ncs_apply_KT", _I, [_P, _P, _P]),
    ("ncs_apply_K_bf16", _I, [_P, _P, _P]),
    ("ncs_apply_KT_bf16", _I, [_P, _P, _P]),
    ("ncs_apply_D", _I, [_P, _P, _P]),
    ("ncs_apply_DT", _I, [_P, _P, _P]),
    ("ncs_apply_Minv", _I, [_P, _P, _P]),
    ("ncs_objective", _I, [_P, _P, _P, _P, _DP]),
    ("ncs_get_mu", _I, [_P, _DP]),
    ("ncs_plan_sizes", _I, [_P, _IP, _IP, _IP]),
    ("ncs_status_string", ctypes.c_char_p, [_I]),
    ("ncs_profile_enable", _I, [_P, _I]),
    ("ncs_profile_enable_mask", _I, [_P, ctypes.c_uint]),
    ("ncs_profile_read", _I, [_P, _DP, _IP, _IP]),
    ("ncs_kernel_name", ctypes.c_char_p, [_I]),
    ("ncs_plan_nnz", _I, [_P, _DP]),
    ("ncs_apply_KT_static", _I, [ctypes.POINTER(Geometry), _I, _P, _P, _P]),
    ("ncs_plan_info", _I, [_P, _IP, _IP, _IP]),
    ("ncs_plan_fwd_strips", _I, [_P, _IP, _IP]),
    ("ncs_fbp", _I, [_P, _P, _P]),
    ("ncs_unet_create", _I, [_I, _I, _I, _I, ctypes.c_uint64, ctypes.POINTER(_P)]),
    ("ncs_unet_destroy", None, [_P]),
    ("ncs_unet_num_params", ctypes.c_size_t, [_P]),
    ("ncs_unet_params", _I, [_P, ctypes.POINTER(ctypes.c_float), _I]),
    ("ncs_unet_forward", _I, [_P, _P, _P]),
    ("ncs_unet_gradient", _I, [_P, _P, _P, _DP, ctypes.POINTER(ctypes.c_float)]),
    ("ncs_unet_train_step", _I, [_P, _P, _P, ctypes.c_float, _DP]),
    ("ncs_unet_set_conv_path", _I, [_P, _I]),
    ("ncs_unet_inject_wait_timeout", _I, [_P]),
    ("ncs_cone_create", _I, [ctypes.POINTER(ConeGeometry), _I, _I, _P, ctypes.POINTER(_P)]),
    ("ncs_cone_destroy", None, [_P]),
    ("ncs_cone_apply_K", _I, [_P, _P, _P]),
    ("ncs_cone_apply_KT", _I, [_P, _P, _P]),
    ("ncs_cone_plan_create", _I, [ctypes.POINTER(ConeGeometry), _I, _I, _D, _D, ctypes.POINTER(Options),
                                  ctypes.POINTER(_P)]),
    ("ncs_cone_plan_destroy", None, [_P]),
    ("ncs_cone_step", _I, [_P, _P, _P, _P, _P, _I]),
    ("ncs_cone_solve", _I, [_P, _P, _P, _D, _I, _D, ctypes.POINTER(Report)]),
    ("ncs_cone_objective", _I, [_P, _P, _P, _DP]),
    ("ncs_cone_kernels", _I, [_P, ctypes.POINTER(ctypes.c_longlong)]),
    ("ncs_cone_apply_Minv", _I, [_P, _P, _P]),
    ("ncs_cone_get_mu", _I, [_P, _DP]),
    ("ncs_cone_power_bound", _I, [_P, _DP]),
    ("ncs_batch_create", _I, [ctypes.POINTER(_P), _I, ctypes.POINTER(_P)]),
    ("ncs_batch_destroy", None, [_P]),
    ("ncs_batch_set_lanes", _I, [_P, _I]),
    ("ncs_batch_tune_lanes", _I, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P), _I,
                                  ctypes.POINTER(_I)]),
    ("ncs_batch_solve", _I, [_P, ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(_P), _D, _I, _DP,
                             ctypes.POINTER(Report)]),
]

NCS_KERNEL_COUNT = 8


def load_library(path: str | None = None) -> ctypes.CDLL:
    """Load libncs.so (built in-tree by __graft_entry__.build() or
    paper_1810_13100_gb300._build.build()).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError("libncs.so is not built (%s); run `python -c 'import __graft_entry__ as g; g.build()'`"
                           % path)
    L = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def status_string(code: int) -> str:
    try:
        return load_library().ncs_status_string(code).decode()
    except Exception:  # library missing
        return "status %d" % code


def _check(code, what):
    if code < 0:
        raise NCSError(code, what)
    return code


def _ptr(t, name, numel=None, allow_none=False, dtype=None):
    """Device pointer of a contiguous CUDA tensor of the given dtype (default
    float32; None -> NULL)."""
    if t is None:
        if allow_none:
            return None
        raise ValueError("%s is required" % name)
    import torch
    dtype = torch.float32 if dtype is None else dtype
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError("%s must be a contiguous %s tensor" % (name, dtype))
    if numel is not None and t.numel() != numel:
        raise ValueError("%s has %d elements, expected %d" % (name, t.numel(), numel))
    return ctypes.c_void_p(t.data_ptr())


def default_options() -> Options:
    o = Options()
    load_library().ncs_options_default(ctypes.byref(o))
    return o


class Plan:
    """An NCS plan: geometry, image side N, TV weight lam, dual step alpha and the
    options of include/ncs.h.  Work runs on `stream` (a torch.cuda.Stream, a raw
    cudaStream_t int, or None for a side stream ordered with torch's current stream).

    Parallel beam by default (ncs_plan_create: n_angles angles, n_det bins, det_spacing,
    det_offset, angles).  Giving src_dist selects the fan beam (ncs_plan_create_fan):
    n_angles source positions (angles: their beta_a, default 2 pi a / n_angles), n_det
    channels at fan pitch fan_pitch (radians) with centre offset fan_offset; fan_gather picks
    its K^T kernel ("auto" / "lines": ray-driven tiles, "quads": pixel-driven 2 x 2 quads).
    fwd_kernel picks the parallel beam's K kernel: "auto" / "strips": image strips staged in
    shared memory, "rows": the row walk ("auto" takes the row walk where strips do not fit)."""

    def __init__(self, N, n_angles, n_det, lam, alpha, *, beta=None, gamma=0.0, h_dc=None, c_r=None,
                 kappa=1.0, data="l2", tv="aniso", nonneg=False, precision="fp32", a3_margin=1e-2,
                 power_max_iter=500, power_tol=1e-6, power_seed=0, check_every=10,
                 det_spacing=1.0, det_offset=0.0, angles=None, stream=None, autotune=False, warm_dual=False,
                 h_probes=0, src_dist=None, fan_pitch=None, fan_offset=0.0, fan_gather="auto", pdhg_only=False,
                 fwd_kernel="auto"):
        import torch
        L = load_library()
        self._L = L
        self.fan = src_dist is not None
        self._angles = None
        arr = None
        if angles is not None:
            arr = (ctypes.c_double * len(angles))(*[float(a) for a in angles])
            self._angles = arr
        if self.fan:
            if fan_pitch is None:
                raise ValueError("a fan-beam plan needs fan_pitch")
            g = FanGeometry()
            g.n_views, g.n_det = int(n_angles), int(n_det)
            g.src_dist, g.pitch, g.offset = float(src_dist), float(fan_pitch), float(fan_offset)
            if arr is not None:
                g.views = ctypes.cast(arr, _DP)
        else:
            g = Geometry()
            g.n_angles, g.n_det = int(n_angles), int(n_det)
            g.det_spacing, g.det_offset = float(det_spacing), float(det_offset)
            if arr is not None:
                g.angles = ctypes.cast(arr, _DP)
        o = default_options()
        nan = float("nan")
        o.beta = nan if beta is None else float(beta)
        o.gamma = float(gamma)
        o.h_dc = nan if h_dc is None else float(h_dc)
        o.c_r = nan if c_r is None else float(c_r)
        o.kappa = float(kappa)
        o.data = {"l2": 0, "kl": 1}[data]
        o.tv = {"aniso": 0, "iso": 1}[tv]
        o.nonneg = 1 if nonneg else 0
        o.prec = {"fp32": 0, "bf16": 1, "bf16-duals": 2}[precision]
        o.a3_margin = float(a3_margin)
        o.power_max_iter = int(power_max_iter)
        o.power_tol = float(power_tol)
        o.power_seed = int(power_seed)
        o.check_every = int(check_every)
        o.autotune = 1 if autotune else 0
        o.warm_dual = 1 if warm_dual else 0
        o.h_probes = int(h_probes)
        o.fan_gather = {"auto": 0, "quads": 1, "lines": 2}[fan_gather]
        o.pdhg_only = 1 if pdhg_only else 0
        o.fwd_kernel = {"auto": 0, "rows": 1, "strips": 2}[fwd_kernel]
        # With no stream given, the plan runs on a side stream that is ordered
        # after torch's current stream on entry to every call and before it on
        # exit, so results are visible to torch without extra synchronisation.
        self._auto = stream is None
        if stream is None:
            stream = torch.cuda.Stream()
        o.cuda_stream = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        self.stream = stream
        h = ctypes.c_void_p()
        if self.fan:
            _check(L.ncs_plan_create_fan(ctypes.byref(g), int(N), int(N), float(lam), float(alpha), ctypes.byref(o),
                                         ctypes.byref(h)), "ncs_plan_create_fan")
        else:
            _check(L.ncs_plan_create(ctypes.byref(g), int(N), int(N), float(lam), float(alpha), ctypes.byref(o),
                                     ctypes.byref(h)), "ncs_plan_create")
        self._h = h
        self.N, self.n_angles, self.n_det = int(N), int(n_angles), int(n_det)
        self.lam, self.alpha = float(lam), float(alpha)
        self.beta = float(alpha if beta is None else beta)
        self.data, self.tv, self.nonneg = data, tv, bool(nonneg)
        # dtype of the duals u, v, s in step (x, b, bg are always float32)
        self.state_dtype = torch.float32 if precision == "fp32" else torch.bfloat16

    def _enter(self):
        if self._auto:
            import torch
            self.stream.wait_stream(torch.cuda.current_stream())

    def _leave(self):
        if self._auto:
            import torch
            torch.cuda.current_stream().wait_stream(self.stream)

    def _call(self, what, fn, *args):
        self._enter()
        try:
            return _check(fn(*args), what)
        finally:
            self._leave()

    # -------------------------------------------------------------- sizes
    @property
    def n(self):
        return self.N * self.N

    @property
    def m(self):
        return self.n_angles * self.n_det

    def close(self):
        if getattr(self, "_h", None):
            self._L.ncs_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -------------------------------------------------------------- iterations
    def _state_ptrs(self, x, u, v, s, b, bg):
        d = self.state_dtype
        return (_ptr(x, "x", self.n), _ptr(u, "u", self.m, dtype=d), _ptr(v, "v", 2 * self.n, dtype=d),
                _ptr(s, "s", self.n, allow_none=True, dtype=d), _ptr(b, "b", self.m),
                _ptr(bg, "bg", self.m, allow_none=True))

    def step(self, x, u, v, s, b, bg=None, n_iter=1):
        """n_iter NCS iterations in place on (x, u, v, s)."""
        self._call("ncs_step", self._L.ncs_step, self._h, *self._state_ptrs(x, u, v, s, b, bg), int(n_iter))

    def pdhg_step(self, x, u, v, s, b, bg=None, n_iter=1):
        self._call("pdhg_step", self._L.pdhg_step, self._h, *self._state_ptrs(x, u, v, s, b, bg), int(n_iter))

    def _solve(self, fn, what, b, x, tol, max_iter, f_star, bg):
        rep = Report()
        self._call(what, fn, self._h, _ptr(b, "b", self.m), _ptr(bg, "bg", self.m, allow_none=True),
                   _ptr(x, "x", self.n), float(tol), int(max_iter), float("nan") if f_star is None else float(f_star),
                   ctypes.byref(rep))
        return rep.as_dict()

    def solve(self, b, x, tol=1e-4, max_iter=2000, f_star=None, bg=None):
        """NCS from x (in/out) with zero duals to the tolerance; returns the report dict."""
        return self._solve(self._L.ncs_solve, "ncs_solve", b, x, tol, max_iter, f_star, bg)

    def pdhg_solve(self, b, x, tol=1e-4, max_iter=2000, f_star=None, bg=None):
        return self._solve(self._L.pdhg_solve, "pdhg_solve", b, x, tol, max_iter, f_star, bg)

    def admm_solve(self, b, x, tol=1e-4, max_outer=500, n_cg=10, f_star=None):
        """The ADMM comparator with a PCG inner loop (admm_solve); x is x^0 in, result out."""
        rep = Report()
        self._call("admm_solve", self._L.admm_solve, self._h, _ptr(b, "b", self.m), _ptr(x, "x", self.n), float(tol),
                   int(max_outer), int(n_cg), float("nan") if f_star is None else float(f_star), ctypes.byref(rep))
        return rep.as_dict()

    def power_bound(self):
        lm, rho = ctypes.c_double(), ctypes.c_double()
        self._call("ncs_power_bound", self._L.ncs_power_bound, self._h, ctypes.byref(lm), ctypes.byref(rho))
        return lm.value, rho.value

    # -------------------------------------------------------------- operators
    def _out(self, out, numel, like):
        import torch
        if out is None:
            out = torch.empty(numel, dtype=torch.float32, device=like.device)
        return out

    def apply_K(self, x, y=None):
        y = self._out(y, self.m, x)
        self._call("ncs_apply_K", self._L.ncs_apply_K, self._h, _ptr(x, "x", self.n), _ptr(y, "y", self.m))
        return y

    def apply_KT(self, y, x=None):
        x = self._out(x, self.n, y)
        self._call("ncs_apply_KT", self._L.ncs_apply_KT, self._h, _ptr(y, "y", self.m), _ptr(x, "x", self.n))
        return x

    def apply_K_bf16(self, x, y=None):
        """K x through bfloat16 pair images of x (ncs_apply_K_bf16); float32 in and out."""
        y = self._out(y, self.m, x)
        self._call("ncs_apply_K_bf16", self._L.ncs_apply_K_bf16, self._h, _ptr(x, "x", self.n),
                   _ptr(y, "y", self.m))
        return y

    def apply_KT_bf16(self, y, x=None):
        """K^T y of a bfloat16 sinogram y (ncs_apply_KT_bf16); float32 out."""
        import torch
        x = self._out(x, self.n, y)
        self._call("ncs_apply_KT_bf16", self._L.ncs_apply_KT_bf16, self._h,
                   _ptr(y, "y", self.m, dtype=torch.bfloat16), _ptr(x, "x", self.n))
        return x

    def apply_D(self, x, v=None):
        v = self._out(v, 2 * self.n, x)
        self._call("ncs_apply_D", self._L.ncs_apply_D, self._h, _ptr(x, "x", self.n), _ptr(v, "v", 2 * self.n))
        return v

    def apply_DT(self, v, x=None):
        x = self._out(x, self.n, v)
        self._call("ncs_apply_DT", self._L.ncs_apply_DT, self._h, _ptr(v, "v", 2 * self.n), _ptr(x, "x", self.n))
        return x

    def fbp(self, b, x=None):
        """Ram-Lak filtered backprojection of the sinogram b."""
        x = self._out(x, self.n, b)
        self._call("ncs_fbp", self._L.ncs_fbp, self._h, _ptr(b, "b", self.m), _ptr(x, "x", self.n))
        return x

    def apply_Minv(self, r, out=None):
        out = self._out(out, self.n, r)
        self._call("ncs_apply_Minv", self._L.ncs_apply_Minv, self._h, _ptr(r, "r", self.n), _ptr(out, "out", self.n))
        return out

    def objective(self, x, b, bg=None):
        f = ctypes.c_double()
        self._call("ncs_objective", self._L.ncs_objective, self._h, _ptr(x, "x", self.n), _ptr(b, "b", self.m),
                   _ptr(bg, "bg", self.m, allow_none=True), ctypes.byref(f))
        return f.value

    def profile(self, on=True):
        """Turn per-kernel CUDA-event timing on or off (clears the record)."""
        self._call("ncs_profile_enable", self._L.ncs_profile_enable, self._h, 1 if on else 0)

    def profile_mask(self, classes):
        """Time only the named kernel classes (ncs_kernel_name names); clears the record."""
        mask = 0
        for k in range(NCS_KERNEL_COUNT):
            if self._L.ncs_kernel_name(k).decode() in classes:
                mask |= 1 << k
        self._call("ncs_profile_enable_mask", self._L.ncs_profile_enable_mask, self._h, mask)

    def profile_read(self):
        """{kernel class: (total ms, launches)} since the last read, then cleared; the CUDA
        kernels those launches enqueued go to self.kernel_launches ({kernel class: count})."""
        ms = (ctypes.c_double * NCS_KERNEL_COUNT)()
        n = (ctypes.c_int * NCS_KERNEL_COUNT)()
        nk = (ctypes.c_int * NCS_KERNEL_COUNT)()
        self._call("ncs_profile_read", self._L.ncs_profile_read, self._h, ms, n, nk)
        names = [self._L.ncs_kernel_name(k).decode() for k in range(NCS_KERNEL_COUNT)]
        self.kernel_launches = {names[k]: nk[k] for k in range(NCS_KERNEL_COUNT)}
        return {names[k]: (ms[k], n[k]) for k in range(NCS_KERNEL_COUNT)}

    def nnz(self):
        """Nonzero weights of K (2 * nnz flops per application of K or K^T)."""
        v = ctypes.c_double()
        _check(self._L.ncs_plan_nnz(self._h, ctypes.byref(v)), "ncs_plan_nnz")
        return v.value

    def info(self):
        """{"gather_parts": int, "fft_radices": [int, ...]} chosen for this plan."""
        gp, nr = ctypes.c_int(), ctypes.c_int()
        rad = (ctypes.c_int * 12)()
        _check(self._L.ncs_plan_info(self._h, ctypes.byref(gp), rad, ctypes.byref(nr)), "ncs_plan_info")
        return {"gather_parts": gp.value, "fft_radices": [rad[k] for k in range(nr.value)]}

    def fwd_strips(self):
        """(strips, rows per strip) of the strip form of K, or (0, 0) for the row walk."""
        ns, nr = ctypes.c_int(), ctypes.c_int()
        _check(self._L.ncs_plan_fwd_strips(self._h, ctypes.byref(ns), ctypes.byref(nr)), "ncs_plan_fwd_strips")
        return ns.value, nr.value

    def mu(self):
        import numpy as np
        out = np.empty(self.n, dtype=np.float64)
        _check(self._L.ncs_get_mu(self._h, out.ctypes.data_as(_DP)), "ncs_get_mu")
        return out.reshape(self.N, self.N)


class Cone:
    """Cone-beam operator pair (ncs_cone_create): K and its exact transpose for an N x N x Nz
    volume.  Work runs on `stream` (torch.cuda.Stream / raw cudaStream_t int / None: a side
    stream ordered with torch's current stream)."""

    def __init__(self, N, Nz, n_views, n_rows, n_det, src_dist, pitch, row_pitch, offset=0.0, row_offset=0.0,
                 views=None, stream=None):
        import torch
        L = load_library()
        self._L = L
        g = ConeGeometry()
        g.n_views, g.n_rows, g.n_det = int(n_views), int(n_rows), int(n_det)
        g.src_dist, g.pitch, g.offset = float(src_dist), float(pitch), float(offset)
        g.row_pitch, g.row_offset = float(row_pitch), float(row_offset)
        self._views = None
        if views is not None:
            self._views = (ctypes.c_double * len(views))(*[float(v) for v in views])
            g.views = ctypes.cast(self._views, _DP)
        self._auto = stream is None
        if stream is None:
            stream = torch.cuda.Stream()
        self.stream = stream
        h = ctypes.c_void_p()
        _check(L.ncs_cone_create(ctypes.byref(g), int(N), int(Nz),
                                 ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)),
                                 ctypes.byref(h)), "ncs_cone_create")
        self._h = h
        self.N, self.Nz = int(N), int(Nz)
        self.n = self.N * self.N * self.Nz
        self.m = int(n_views) * int(n_rows) * int(n_det)

    def _call(self, what, fn, *args):
        import torch
        if self._auto:
            self.stream.wait_stream(torch.cuda.current_stream())
        try:
            return _check(fn(*args), what)
        finally:
            if self._auto:
                torch.cuda.current_stream().wait_stream(self.stream)

    def apply_K(self, x, y=None):
        import torch
        y = torch.empty(self.m, device=x.device) if y is None else y
        self._call("ncs_cone_apply_K", self._L.ncs_cone_apply_K, self._h, _ptr(x, "x", self.n), _ptr(y, "y", self.m))
        return y

    def apply_KT(self, y, x=None):
        import torch
        x = torch.empty(self.n, device=y.device) if x is None else x
        self._call("ncs_cone_apply_KT", self._L.ncs_cone_apply_KT, self._h, _ptr(y, "y", self.m), _ptr(x, "x", self.n))
        return x

    def close(self):
        if getattr(self, "_h", None):
            self._L.ncs_cone_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ConePlan:
    """3-D cone-beam NCS (ncs_cone_plan_create): N x N x Nz volume, TV-CT with L2 data.  The
    geometry arguments are those of Cone; lam, alpha and the keyword options those of Plan
    (beta, gamma, h_dc, tv, h_probes (0 -> 128), a3_margin, power_*, check_every).  Work runs
    on a side stream ordered with torch's current stream."""

    def __init__(self, N, Nz, n_views, n_rows, n_det, src_dist, pitch, row_pitch, lam, alpha, *, offset=0.0,
                 row_offset=0.0, views=None, beta=None, gamma=0.0, h_dc=None, tv="aniso", h_probes=0,
                 a3_margin=1e-2, power_max_iter=500, power_tol=1e-6, power_seed=0, check_every=10):
        import torch
        L = load_library()
        self._L = L
        g = ConeGeometry()
        g.n_views, g.n_rows, g.n_det = int(n_views), int(n_rows), int(n_det)
        g.src_dist, g.pitch, g.offset = float(src_dist), float(pitch), float(offset)
        g.row_pitch, g.row_offset = float(row_pitch), float(row_offset)
        self._views = None
        if views is not None:
            self._views = (ctypes.c_double * len(views))(*[float(v) for v in views])
            g.views = ctypes.cast(self._views, _DP)
        o = default_options()
        nan = float("nan")
        o.beta = nan if beta is None else float(beta)
        o.gamma = float(gamma)
        o.h_dc = nan if h_dc is None else float(h_dc)
        o.tv = {"aniso": 0, "iso": 1}[tv]
        o.h_probes = int(h_probes)
        o.a3_margin = float(a3_margin)
        o.power_max_iter = int(power_max_iter)
        o.power_tol = float(power_tol)
        o.power_seed = int(power_seed)
        o.check_every = int(check_every)
        self.stream = torch.cuda.Stream()
        o.cuda_stream = self.stream.cuda_stream
        h = ctypes.c_void_p()
        _check(L.ncs_cone_plan_create(ctypes.byref(g), int(N), int(Nz), float(lam), float(alpha), ctypes.byref(o),
                                      ctypes.byref(h)), "ncs_cone_plan_create")
        self._h = h
        self.N, self.Nz = int(N), int(Nz)
        self.n = self.N * self.N * self.Nz
        self.m = int(n_views) * int(n_rows) * int(n_det)

    def _call(self, what, fn, *args):
        import torch
        self.stream.wait_stream(torch.cuda.current_stream())
        try:
            return _check(fn(*args), what)
        finally:
            torch.cuda.current_stream().wait_stream(self.stream)

    def step(self, x, u, v, b, n_iter=1):
        self._call("ncs_cone_step", self._L.ncs_cone_step, self._h, _ptr(x, "x", self.n), _ptr(u, "u", self.m),
                   _ptr(v, "v", 3 * self.n), _ptr(b, "b", self.m), int(n_iter))

    def solve(self, b, x, tol=1e-4, max_iter=2000, f_star=None):
        rep = Report()
        code = self._call("ncs_cone_solve", self._L.ncs_cone_solve, self._h, _ptr(b, "b", self.m),
                          _ptr(x, "x", self.n), float(tol), int(max_iter),
                          float("nan") if f_star is None else float(f_star), ctypes.byref(rep))
        out = rep.as_dict()
        out["code"] = code
        return out

    def objective(self, x, b):
        f = ctypes.c_double()
        self._call("ncs_cone_objective", self._L.ncs_cone_objective, self._h, _ptr(x, "x", self.n),
                   _ptr(b, "b", self.m), ctypes.byref(f))
        return f.value

    def kernels(self):
        """CUDA kernels the plan has enqueued since creation (a solve's graph counts once)."""
        n = ctypes.c_longlong()
        _check(self._L.ncs_cone_kernels(self._h, ctypes.byref(n)), "ncs_cone_kernels")
        return n.value

    def apply_Minv(self, r, out=None):
        import torch
        out = torch.empty(self.n, device=r.device) if out is None else out
        self._call("ncs_cone_apply_Minv", self._L.ncs_cone_apply_Minv, self._h, _ptr(r, "r", self.n),
                   _ptr(out, "out", self.n))
        return out

    def mu(self):
        import numpy as np
        out = np.empty(self.n, dtype=np.float64)
        _check(self._L.ncs_cone_get_mu(self._h, out.ctypes.data_as(_DP)), "ncs_cone_get_mu")
        return out.reshape(self.Nz, self.N, self.N)

    def power_bound(self):
        rho = ctypes.c_double()
        _check(self._L.ncs_cone_power_bound(self._h, ctypes.byref(rho)), "ncs_cone_power_bound")
        return rho.value

    def close(self):
        if getattr(self, "_h", None):
            self._L.ncs_cone_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent slices solved together (ncs_batch_solve): one CUDA graph with a
    branch per active slice per launch.  `plans` are Plan objects with distinct
    streams; they must outlive the batch."""

    def __init__(self, plans):
        L = load_library()
        self._L = L
        self.plans = list(plans)
        arr = (_P * len(self.plans))(*[p._h.value for p in self.plans])
        h = ctypes.c_void_p()
        _check(L.ncs_batch_create(arr, len(self.plans), ctypes.byref(h)), "ncs_batch_create")
        self._h = h

    def set_lanes(self, lanes):
        """At most `lanes` slices in flight at once (0 = all)."""
        _check(self._L.ncs_batch_set_lanes(self._h, int(lanes)), "ncs_batch_set_lanes")

    def tune_lanes(self, bs, xs, iters=20, bgs=None):
        """Pick the fastest lane count by timed solves (ncs_batch_tune_lanes); xs are
        overwritten.  Returns the lane count."""
        n = len(self.plans)
        for p in self.plans:
            p._enter()
        bp = (_P * n)(*[_ptr(b, "b", p.m).value for b, p in zip(bs, self.plans)])
        xp = (_P * n)(*[_ptr(x, "x", p.n).value for x, p in zip(xs, self.plans)])
        gp = None
        if bgs is not None:
            gp = (_P * n)(*[(_ptr(g, "bg", p.m).value if g is not None else None) for g, p in zip(bgs, self.plans)])
        lanes = ctypes.c_int()
        code = self._L.ncs_batch_tune_lanes(self._h, bp, gp, xp, int(iters), ctypes.byref(lanes))
        for p in self.plans:
            p._leave()
        _check(code, "ncs_batch_tune_lanes")
        return lanes.value

    def close(self):
        if getattr(self, "_h", None):
            self._L.ncs_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, bs, xs, tol=1e-4, max_iter=2000, f_stars=None, bgs=None):
        """Solve every slice; bs, xs (and bgs) are lists of CUDA tensors.  Returns
        (status, [report dict per slice])."""
        import torch
        n = len(self.plans)
        for p in self.plans:
            p._enter()
        bp = (_P * n)(*[_ptr(b, "b", p.m).value for b, p in zip(bs, self.plans)])
        xp = (_P * n)(*[_ptr(x, "x", p.n).value for x, p in zip(xs, self.plans)])
        gp = None
        if bgs is not None:
            gp = (_P * n)(*[(_ptr(g, "bg", p.m).value if g is not None else None) for g, p in zip(bgs, self.plans)])
        fs = None
        if f_stars is not None:
            fs = (ctypes.c_double * n)(*[float("nan") if v is None else float(v) for v in f_stars])
        reps = (Report * n)()
        code = self._L.ncs_batch_solve(self._h, bp, gp, xp, float(tol), int(max_iter), fs, reps)
        for p in self.plans:
            p._leave()
        _check(code, "ncs_batch_solve")
        return code, [r.as_dict() for r in reps]


class UNet:
    """The warm-start U-Net of include/ncs.h (y = x + net(x)) for H x W images."""

    def __init__(self, H, W, levels=4, base=32, seed=0):
        L = load_library()
        self._L = L
        h = ctypes.c_void_p()
        _check(L.ncs_unet_create(int(H), int(W), int(levels), int(base), int(seed), ctypes.byref(h)),
               "ncs_unet_create")
        self._h = h
        self.H, self.W, self.levels, self.base = int(H), int(W), int(levels), int(base)
        self.n_params = int(L.ncs_unet_num_params(h))

    def close(self):
        if getattr(self, "_h", None):
            self._L.ncs_unet_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        import numpy as np
        out = np.empty(self.n_params, dtype=np.float32)
        _check(self._L.ncs_unet_params(self._h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), 0),
               "ncs_unet_params")
        return out

    def set_params(self, p):
        import numpy as np
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.n_params
        _check(self._L.ncs_unet_params(self._h, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), 1),
               "ncs_unet_params")

    def forward(self, x, y=None):
        import torch
        torch.cuda.current_stream().synchronize()
        y = torch.empty(self.H * self.W, dtype=torch.float32, device=x.device) if y is None else y
        _check(self._L.ncs_unet_forward(self._h, _ptr(x, "x", self.H * self.W), _ptr(y, "y", self.H * self.W)),
               "ncs_unet_forward")
        return y

    def gradient(self, x, target):
        import numpy as np
        import torch
        torch.cuda.current_stream().synchronize()
        g = np.empty(self.n_params, dtype=np.float32)
        loss = ctypes.c_double()
        _check(self._L.ncs_unet_gradient(self._h, _ptr(x, "x", self.H * self.W), _ptr(target, "t", self.H * self.W),
                                         ctypes.byref(loss), g.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
               "ncs_unet_gradient")
        return loss.value, g

    def inject_wait_timeout(self):
        """Failure-path test: the next forward / gradient / train step returns NCS_ERR_TIMEOUT."""
        _check(self._L.ncs_unet_inject_wait_timeout(self._h), "ncs_unet_inject_wait_timeout")

    def set_conv_path(self, tensor_cores=True):
        """tcgen05 tensor-core convolutions (True, the default) or the mma.sync path (False)."""
        _check(self._L.ncs_unet_set_conv_path(self._h, 1 if tensor_cores else 0), "ncs_unet_set_conv_path")

    def train_step(self, x, target, lr):
        import torch
        torch.cuda.current_stream().synchronize()
        loss = ctypes.c_double()
        _check(self._L.ncs_unet_train_step(self._h, _ptr(x, "x", self.H * self.W), _ptr(target, "t", self.H * self.W),
                                           float(lr), ctypes.byref(loss)), "ncs_unet_train_step")
        return loss.value
