"""Seeded ellipse phantoms, their exact parallel-beam line integrals, and noise.

Recipe (the stand-in for the paper's patient / XCAT / PET data of Sec. 5, which
are not available): x_true is a sum of random ellipses in a [-1, 1]^2 frame,
rasterised at the pixel centres and rounded to float32; the measured data are
b = K x_true + Gaussian noise (CT, sigma = a fraction of max(K x_true)) or a
Poisson draw with mean s K x_true + r (PET).  K is the CALLER's projector (this
module holds none): the tests pass the FP64 oracle's, the benchmark the
library's.  The exact line integrals of the ellipses (`radon_ellipses`) serve
the tests that pin the projector.  Every returned array is rounded once to
float32 so the GPU path and the FP64 oracle consume identical values.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class Ellipses:
    """Ellipse parameters in the normalised frame [-1, 1]^2 (one row per ellipse).

    cx, cy: centre; ax, ay: semi-axes; phi: rotation of the ax-axis from +u;
    rho: additive intensity.
    """
    cx: np.ndarray
    cy: np.ndarray
    ax: np.ndarray
    ay: np.ndarray
    phi: np.ndarray
    rho: np.ndarray

    def __len__(self):
        return len(self.cx)


def draw_ellipses(rng: np.random.Generator, n: int) -> Ellipses:
    """Draw n ellipses: centres U[-0.8,0.8]^2, semi-axes U[0.05,0.5], rotation
    U[0,pi), intensity U[0,1].  The draw order is fixed (centres, axes,
    rotations, intensities) so a seed always gives the same phantom."""
    c = rng.uniform(-0.8, 0.8, size=(n, 2))
    ax = rng.uniform(0.05, 0.5, size=(n, 2))
    phi = rng.uniform(0.0, math.pi, size=n)
    rho = rng.uniform(0.0, 1.0, size=n)
    return Ellipses(c[:, 0].copy(), c[:, 1].copy(), ax[:, 0].copy(), ax[:, 1].copy(), phi, rho)


def _pixel_grid(N: int):
    """Normalised coordinates of the pixel centres, arrays of shape (N, N)."""
    idx = np.arange(N, dtype=np.float64)
    u = (idx - (N - 1) / 2.0) * (2.0 / N)          # columns, left to right
    v = ((N - 1) / 2.0 - idx) * (2.0 / N)          # rows, top to bottom
    U, V = np.meshgrid(u, v)                       # U[j, i] = u_i, V[j, i] = v_j
    return U, V


def rasterize(ell: Ellipses, N: int) -> np.ndarray:
    """Pixel value = sum of the intensities of the ellipses that contain the
    pixel centre (float64, shape (N, N))."""
    U, V = _pixel_grid(N)
    img = np.zeros((N, N), dtype=np.float64)
    for k in range(len(ell)):
        du, dv = U - ell.cx[k], V - ell.cy[k]
        c, s = math.cos(ell.phi[k]), math.sin(ell.phi[k])
        p = (du * c + dv * s) / ell.ax[k]
        q = (-du * s + dv * c) / ell.ay[k]
        img += np.where(p * p + q * q <= 1.0, ell.rho[k], 0.0)
    return img


@dataclasses.dataclass(frozen=True)
class Ellipsoids:
    """Ellipsoid parameters in the normalised frame [-1, 1]^3 (one row per ellipsoid): centre,
    semi-axes, rotation phi about the w axis, additive intensity."""
    c: np.ndarray      # (n, 3)
    ax: np.ndarray     # (n, 3)
    phi: np.ndarray
    rho: np.ndarray


def draw_ellipsoids(rng: np.random.Generator, n: int) -> Ellipsoids:
    """Draw n ellipsoids: centres U[-0.8,0.8]^3, semi-axes U[0.05,0.5]^3, rotation about w
    U[0,pi), intensity U[0,1], in that fixed order."""
    c = rng.uniform(-0.8, 0.8, size=(n, 3))
    ax = rng.uniform(0.05, 0.5, size=(n, 3))
    phi = rng.uniform(0.0, math.pi, size=n)
    rho = rng.uniform(0.0, 1.0, size=n)
    return Ellipsoids(c, ax, phi, rho)


def rasterize3(ell: Ellipsoids, N: int, Nz: int) -> np.ndarray:
    """Voxel value = sum of the intensities of the ellipsoids that contain the voxel centre
    (float64, shape (Nz, N, N)); the volume spans [-1, 1] along each axis."""
    U, V = _pixel_grid(N)
    w = ((np.arange(Nz, dtype=np.float64) - (Nz - 1) / 2.0) * (2.0 / Nz))[:, None, None]
    vol = np.zeros((Nz, N, N), dtype=np.float64)
    for k in range(len(ell.rho)):
        du, dv, dw = U[None] - ell.c[k, 0], V[None] - ell.c[k, 1], w - ell.c[k, 2]
        c, s = math.cos(ell.phi[k]), math.sin(ell.phi[k])
        p = (du * c + dv * s) / ell.ax[k, 0]
        q = (-du * s + dv * c) / ell.ax[k, 1]
        r = dw / ell.ax[k, 2]
        vol += np.where(p * p + q * q + r * r <= 1.0, ell.rho[k], 0.0)
    return vol


def ct3d_problem(seed: int, N: int, Nz: int, n_views: int, n_rows: int, n_det: int, n_ellipsoids: int,
                 noise_frac: float, project) -> dict:
    """Seeded 3-D TV-CT instance: b = project(x_true) + N(0, sigma^2), sigma = noise_frac *
    max(project(x_true)); `project` maps the float32 volume (Nz, N, N) to its (n_views,
    n_rows, n_det) sinogram.  Draw order: the ellipsoids, then the noise.  Arrays float32."""
    rng = np.random.default_rng(seed)
    ell = draw_ellipsoids(rng, n_ellipsoids)
    x_true = _f32(rasterize3(ell, N, Nz))
    z = rng.standard_normal((n_views, n_rows, n_det))
    b, sigma = ct_data(project(x_true), z, noise_frac)
    return dict(kind="ct", seed=seed, N=N, Nz=Nz, x_true=x_true, b=b, sigma=sigma)


def angles(n_angles: int) -> np.ndarray:
    """theta_a = a*pi/n_angles (float64)."""
    return np.arange(n_angles, dtype=np.float64) * (math.pi / n_angles)


def det_centres(n_det: int, det_spacing: float = 1.0, det_offset: float = 0.0) -> np.ndarray:
    """s_t = (t - (n_det-1)/2)*spacing + offset in pixel units (float64)."""
    return (np.arange(n_det, dtype=np.float64) - (n_det - 1) / 2.0) * det_spacing + det_offset


def radon_ellipses(ell: Ellipses, N: int, theta: np.ndarray, s_pix: np.ndarray) -> np.ndarray:
    """Exact line integrals (pixel units) of the ellipse phantom along the rays
    u cos(theta) + v sin(theta) = s, returned as y[a, t] (float64).

    For one ellipse the chord along a line at signed distance s' from its
    centre is 2*A*B*sqrt(a2 - s'^2)/a2 with a2 = A^2 cos^2(theta-phi) +
    B^2 sin^2(theta-phi) (textbook closed form; checked by brute-force
    sampling in the tests).  Lengths are computed in the normalised frame and
    scaled by N/2 to pixel units.
    """
    th = np.asarray(theta, dtype=np.float64)[:, None]
    s = np.asarray(s_pix, dtype=np.float64)[None, :] * (2.0 / N)
    out = np.zeros((th.shape[0], s.shape[1]), dtype=np.float64)
    for k in range(len(ell)):
        A, B = ell.ax[k], ell.ay[k]
        d = th - ell.phi[k]
        a2 = (A * np.cos(d)) ** 2 + (B * np.sin(d)) ** 2
        sp = s - (ell.cx[k] * np.cos(th) + ell.cy[k] * np.sin(th))
        disc = a2 - sp * sp
        out += np.where(disc > 0.0, 2.0 * ell.rho[k] * A * B * np.sqrt(np.maximum(disc, 0.0)) / a2, 0.0)
    return out * (N / 2.0)


def _f32(a: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))


def ct_phantom(seed: int, N: int, n_angles: int, n_det: int, n_ellipses: int):
    """First half of a CT instance: (x_true as float32 (N, N), z) with z the seeded
    standard normal draws of shape (n_angles, n_det) that become the noise.  Draw
    order: the ellipses, then z."""
    rng = np.random.default_rng(seed)
    ell = draw_ellipses(rng, n_ellipses)
    x_true = _f32(rasterize(ell, N))
    z = rng.standard_normal((n_angles, n_det))
    return x_true, z


def ct_data(Kx: np.ndarray, z: np.ndarray, noise_frac: float):
    """Second half: b = K x_true + sigma z with sigma = noise_frac * max(K x_true),
    rounded to float32.  Returns (b, sigma)."""
    Kx = np.asarray(Kx, dtype=np.float64).reshape(z.shape)
    sigma = noise_frac * float(Kx.max())
    return _f32(Kx + sigma * z), sigma


def ct_problem(seed: int, N: int, n_angles: int, n_det: int, n_ellipses: int,
               noise_frac: float, project, det_spacing: float = 1.0, det_offset: float = 0.0) -> dict:
    """Seeded TV-CT instance: b = project(x_true) + N(0, sigma^2) with
    sigma = noise_frac * max(project(x_true)).  `project` maps the float32 image
    (N, N) to its (n_angles, n_det) sinogram with the given detector spacing and
    offset.  Arrays are float32."""
    x_true, z = ct_phantom(seed, N, n_angles, n_det, n_ellipses)
    b, sigma = ct_data(project(x_true), z, noise_frac)
    return dict(kind="ct", seed=seed, N=N, n_angles=n_angles, n_det=n_det,
                det_spacing=det_spacing, det_offset=det_offset,
                x_true=x_true, b=b, sigma=sigma)


def pet_problem(seed: int, N: int, n_angles: int, n_det: int, n_ellipses: int, project,
                total_counts: float = 1e6, bg_frac: float = 0.1) -> dict:
    """Seeded TV-PET instance: y ~ Poisson(s P + r) with P = project(x_true) of
    the activity phantom, s scaling sum(s P) to total_counts and the uniform
    background r = bg_frac times the mean of s P.  Arrays float32 (x_true is
    returned times s, the image the data measure); r_bg is sinogram-shaped."""
    rng = np.random.default_rng(seed)
    ell = draw_ellipses(rng, n_ellipses)
    x0 = _f32(rasterize(ell, N))
    P = np.asarray(project(x0), dtype=np.float64).reshape(n_angles, n_det)
    scale = total_counts / float(P.sum())
    mean_counts = scale * P
    r = bg_frac * float(mean_counts.mean())
    y = rng.poisson(mean_counts + r).astype(np.float64)
    return dict(kind="pet", seed=seed, N=N, n_angles=n_angles, n_det=n_det,
                det_spacing=1.0, det_offset=0.0,
                x_true=_f32(x0.astype(np.float64) * scale), b=_f32(y),
                r_bg=_f32(np.full_like(y, r)), scale=scale, r=r)


def batch_sides(seed: int, n_slices: int = 64, choices=(256, 384, 512)) -> list:
    """Image sides of the uneven batch, drawn by seed; angles = round(1.4*side),
    bins = side + 2 for each slice."""
    rng = np.random.default_rng(seed)
    sides = rng.choice(np.asarray(choices), size=n_slices)
    return [int(s) for s in sides]


# Named workloads (sizes, regularisation and noise of each synthetic case).
WORKLOADS = {
    # 64x64 TV-CT, anisotropic TV, lambda 0.01, 1% noise, 10 ellipses.
    "ct64": dict(kind="ct", N=64, n_angles=90, n_det=92, n_ellipses=10, noise_frac=0.01,
                 lam=0.01, tv="aniso"),
    # 512x512 TV-CT, isotropic TV, lambda 0.005, 0.5% noise, 20 ellipses.
    "ct512": dict(kind="ct", N=512, n_angles=720, n_det=730, n_ellipses=20, noise_frac=0.005,
                  lam=0.005, tv="iso"),
    # 256x256 TV-PET, 1e6 counts, 10% background, lambda 0.02, nonnegativity.
    "pet256": dict(kind="pet", N=256, n_angles=180, n_det=257, n_ellipses=15,
                   lam=0.02, tv="aniso"),
    # Fan-beam TV-CT (equiangular detector, full turn of source positions): the source at
    # twice the image side from the centre, the fan just covering the image's circumscribed
    # circle (fan_pitch with the given cover).  64x64: 120 views, 96 channels, the 64x64
    # noise and lambda; 512x512: 720 views, 768 channels, the 512x512 noise and lambda.
    "fan64": dict(kind="ct", geometry="fan", N=64, n_angles=120, n_det=96, src_dist=128.0, cover=1.05,
                  n_ellipses=10, noise_frac=0.01, lam=0.01, tv="aniso"),
    "fan512": dict(kind="ct", geometry="fan", N=512, n_angles=720, n_det=768, src_dist=1024.0, cover=1.02,
                   n_ellipses=20, noise_frac=0.005, lam=0.005, tv="iso"),
    # Cone-beam TV-CT (circular orbit, cylindrical detector): 128 x 128 x 32 volume, 180 views
    # on a full turn, 32 rows x 192 channels, source at twice the side, 12 ellipsoids.
    "cone128": dict(kind="ct", geometry="cone", N=128, Nz=32, n_angles=180, n_rows=32, n_det=192,
                    src_dist=256.0, cover=1.05, n_ellipses=12, noise_frac=0.005, lam=0.005, tv="iso"),
    # the same proportions at half the size (64 x 64 x 16, 90 views, 16 rows x 96 channels), small
    # enough for the FP64 oracle to reach a tight reference minimum
    "cone64": dict(kind="ct", geometry="cone", N=64, Nz=16, n_angles=90, n_rows=16, n_det=96,
                   src_dist=128.0, cover=1.05, n_ellipses=8, noise_frac=0.005, lam=0.005, tv="iso"),
}


def cone_row_pitch(N: int, Nz: int, src_dist: float, n_rows: int, cover: float = 1.05) -> float:
    """Slope step between detector rows whose slopes span the volume's top and bottom faces
    seen from the nearest point of its circumscribed cylinder, widened by `cover`."""
    return 2.0 * (Nz / 2.0) / (src_dist - N / math.sqrt(2.0)) * cover / n_rows


def fan_pitch(N: int, src_dist: float, n_det: int, cover: float = 1.02) -> float:
    """Fan angle between adjacent channels (radians) for n_det channels whose fan spans the
    circle circumscribing the N x N image seen from distance src_dist, widened by `cover`."""
    return 2.0 * math.asin(N / math.sqrt(2.0) / src_dist) * cover / n_det
