"""Particle-state kinematics of the Dirac walk (Sec. 5.1, Proposition "dispersive differential
equation", second order): drift vector v_k = grad_k omega_k and diffusion tensor
D_k = grad_k grad_k omega_k.  TEST INFRASTRUCTURE.

omega_k = arccos(n u_k) (Sec. 3.2), so with S = sin omega_k:
    grad omega        = -n grad u / S,
    d_i d_j omega     = -(n d_i d_j u + n u d_i omega d_j omega) / S
(differentiating S' = cos(omega) omega' = n u omega').  The derivatives of u_k are those of
the Weyl symbols (Eqs. weyl1d, weyl2d, weyl3d) written out below; k is the wave number (1D),
the lattice wave numbers (k1, k2) conjugate to the lattice coordinates (a, b) (2D), and the
Cartesian wave vector conjugate to the physical BCC coordinates (3D), i.e. the coordinates of
the position observables.  Undefined where S = 0 (omega = 0 or pi: m = 0 and n~_k = 0).
"""

import numpy as np

from .walk import mass_n

__all__ = ["u_derivatives", "drift", "diffusion"]


def u_derivatives(dim, k):
    """(u, grad u, Hessian of u) at one wave vector k (length dim)."""
    k = np.asarray(k, dtype=float).reshape(dim)
    if dim == 1:
        c, s = np.cos(k[0]), np.sin(k[0])
        return c, np.array([-s]), np.array([[-c]])
    if dim == 2:
        kx, ky = 0.5 * (k[0] + k[1]), 0.5 * (k[0] - k[1])
        cx, cy, sx, sy = np.cos(kx), np.cos(ky), np.sin(kx), np.sin(ky)
        u = cx * cy
        # d/dk1 = (d/dkx + d/dky) / 2, d/dk2 = (d/dkx - d/dky) / 2
        ux, uy = -sx * cy, -cx * sy
        uxx, uyy, uxy = -cx * cy, -cx * cy, sx * sy
        g = 0.5 * np.array([ux + uy, ux - uy])
        H = 0.25 * np.array([[uxx + 2 * uxy + uyy, uxx - uyy],
                             [uxx - uyy, uxx - 2 * uxy + uyy]])
        return u, g, H
    cx, cy, cz = np.cos(k)
    sx, sy, sz = np.sin(k)
    u = cx * cy * cz + sx * sy * sz
    g = np.array([-sx * cy * cz + cx * sy * sz,
                  -cx * sy * cz + sx * cy * sz,
                  -cx * cy * sz + sx * sy * cz])
    hxy = sx * sy * cz + cx * cy * sz
    hxz = sx * cy * sz + cx * sy * cz
    hyz = cx * sy * sz + sx * cy * cz
    H = np.array([[-u, hxy, hxz], [hxy, -u, hyz], [hxz, hyz, -u]])
    return u, g, H


def drift(dim, m, k):
    """v_k = grad_k omega_k."""
    n = mass_n(m)
    u, g, _ = u_derivatives(dim, k)
    S = np.sqrt(max(0.0, 1.0 - (n * u) ** 2))
    return -n * g / S


def diffusion(dim, m, k):
    """D_k = grad_k grad_k omega_k (symmetric dim x dim)."""
    n = mass_n(m)
    u, g, H = u_derivatives(dim, k)
    S = np.sqrt(max(0.0, 1.0 - (n * u) ** 2))
    v = -n * g / S
    return -(n * H + n * u * np.outer(v, v)) / S
