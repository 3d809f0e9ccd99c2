"""Shared helpers for the tests: layout conversions between the library's
device arrays and the oracle's, error measures, and the oracle's projector for
the seeded input generator.  No method arithmetic of their own."""
import numpy as np


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def v_to_oracle(v, N):
    """2*N*N device layout -> (dh (N, N-1), dv (N-1, N))."""
    v = np.asarray(v, dtype=np.float64).reshape(2, N, N)
    return v[0][:, :-1].copy(), v[1][:-1, :].copy()


def v_from_oracle(dh, dv):
    N = dh.shape[0]
    out = np.zeros((2, N, N))
    out[0][:, :-1] = dh
    out[1][:-1, :] = dv
    return out.ravel()


def to_np(t):
    return t.detach().cpu().numpy().astype(np.float64)


def f32(a):
    """Round to float32 and back: the values the GPU sees."""
    return np.asarray(a, dtype=np.float64).astype(np.float32).astype(np.float64)


_MU_CACHE = {}


def oracle_scaled_mu(N, na, nd, alpha, beta, gamma, tv, kappa=0.0, kind="ct"):
    """The oracle's eigenvalues of M after the (A3) rescale, and rho (cached per
    geometry and parameters; the power iteration dominates the oracle's cost)."""
    from oracle import circulant as oci
    from oracle import operators as oop
    from oracle import solvers as osv
    key = (N, na, nd, alpha, beta, gamma, tv, kappa, kind)
    if key not in _MU_CACHE:
        g = oop.Geometry(N, na, nd)
        P = osv.Problem(g, np.zeros((na, nd)), lam=0.0, alpha=alpha, beta=beta, tv=tv, kind=kind,
                        kappa=kappa)
        mu0 = oci.mu_table(g, alpha, beta, gamma, kappa=kappa)
        mus, rho = osv.a3_scaled_mu(P, mu0)
        _MU_CACHE[key] = (mus, rho)
    return _MU_CACHE[key]


def oproj(N, na, nd, spacing=1.0, offset=0.0):
    """The oracle's K for synth.ct_problem / pet_problem (b = K x_true + noise)."""
    from oracle import operators as oop
    return oop.projector(N, na, nd, spacing=spacing, offset=offset)
