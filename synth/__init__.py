"""Seeded synthetic inputs for the NCS workloads (phantoms, sinograms, noise).

This module is shared by the FP64 oracle, the tests and the benchmark.  It holds
none of the method's arithmetic (no discrete projector, no finite differences,
no circulant solve, no proximal map): the measured data b = K x_true + noise are
made with a projector that the caller passes in (the oracle's K in the tests and
in oracle/fstar.py, the library's K in the benchmark and the warm-start
pipeline).

Conventions (the paper's Radon transform, Sec. 2, eq. (radon-def)):
  * image x[j, i], N x N, row-major; pixel centre (u, v) = (i - (N-1)/2, (N-1)/2 - j)
    in pixel units (u to the right, v up);
  * angles theta_a = a*pi/n_angles, a = 0..n_angles-1;
  * detector bin centres s_t = (t - (n_det-1)/2) * det_spacing + det_offset;
  * a ray is the line u cos(theta) + v sin(theta) = s; the sinogram is y[a, t].
"""
from .phantom import (  # noqa: F401
    Ellipses,
    draw_ellipses,
    rasterize,
    radon_ellipses,
    angles,
    det_centres,
    ct_phantom,
    ct_data,
    ct_problem,
    pet_problem,
    WORKLOADS,
    batch_sides,
    fan_pitch,
    cone_row_pitch,
    draw_ellipsoids,
    rasterize3,
    ct3d_problem,
)
