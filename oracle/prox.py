"""FP64 oracle proximal maps.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 2: prox_{a g}(z) = argmin_x a g(x) + 1/2 ||x - z||^2, and Moreau's
identity (eq. (Moreau)) prox_{a g*}(x) = x - a prox_{(1/a) g}(x / a).
"""
from __future__ import annotations

import numpy as np


def prox_l2_conj(z, alpha):
    """prox_{alpha g*} for g = 1/2 ||.||^2 (Sec. 4.1: the CT data update
    divides by 1 + alpha)."""
    return z / (1.0 + alpha)


def clip(z, s):
    """Pi_{[-s, s]} componentwise (Sec. 4.1): prox of the conjugate of s ||.||_1."""
    return np.minimum(np.maximum(z, -s), s)


def ball2(zh, zv, s):
    """Projection of each pixel's 2-vector (zh, zv) onto the l2 ball of radius s:
    prox of the conjugate of s * sum_p ||(zh_p, zv_p)||_2 (isotropic TV, not
    in the paper)."""
    nrm = np.sqrt(zh * zh + zv * zv)
    f = np.where(nrm > s, s / np.where(nrm > 0, nrm, 1.0), 1.0)
    return zh * f, zv * f


def S_kl(u, c):
    """Sec. 4.2: S(u; c) = 1 + (u - 1 - sqrt((u-1)^2 + 4c)) / 2, the prox of
    alpha times the conjugate of l(.; b) with c = alpha*b."""
    return 1.0 + (u - 1.0 - np.sqrt((u - 1.0) ** 2 + 4.0 * c)) / 2.0


def min0(z):
    """Projection onto R_- (prox of the conjugate of the indicator of R_+)."""
    return np.minimum(z, 0.0)


def soft(z, t):
    """prox of t ||.||_1 (soft threshold)."""
    return np.sign(z) * np.maximum(np.abs(z) - t, 0.0)


def soft_iso(zh, zv, t):
    """prox of t * sum_p ||(zh_p, zv_p)||_2 (block soft threshold)."""
    nrm = np.sqrt(zh * zh + zv * zv)
    f = np.maximum(1.0 - t / np.where(nrm > 0, nrm, 1.0), 0.0)
    f = np.where(nrm > 0, f, 0.0)
    return zh * f, zv * f
