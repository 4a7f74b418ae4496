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

The accuracy of that second-order description is the overlap of Eq. overlap: a packet
psi^(k, 0) = g(k) u_+(k) evolves exactly to exp(-i omega_k t) psi^(k, 0), and the truncated
equation (Eq. diff-eq-2) gives exp(-i (omega' + v.K + K.D.K / 2) t) psi^(k, 0) with K = k - k',
so their overlap is |sum_k |g|^2 exp(-i R_k t)| / sum_k |g|^2 with R_k the Taylor remainder
of omega beyond second order; the Proposition bounds it below by 1 - eps - gamma Sigma^3 t
(n = 2) up to O(Sigma^5) t.
"""

import itertools
import math

import numpy as np

from .walk import mass_n

__all__ = ["u_derivatives", "drift", "diffusion", "third_derivatives", "fidelity_bound",
           "drift_diffusion_overlap"]


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


def third_derivatives(dim, m, k, h=1e-5):
    """T[i, j, l] = d_i d_j d_l omega_k at k: central differences (step h) of the analytic
    diffusion tensor above, symmetrised over the index order (error O(h^2))."""
    k = np.asarray(k, dtype=float).reshape(dim)
    T = np.zeros((dim, dim, dim))
    for l in range(dim):
        e = np.zeros(dim)
        e[l] = h
        T[:, :, l] = (diffusion(dim, m, k + e) - diffusion(dim, m, k - e)) / (2.0 * h)
    return sum(np.transpose(T, p) for p in itertools.permutations(range(3))) / 6.0


def fidelity_bound(dim, m, k0, weight, dk, sigma_box, t):
    """Lower bound of the overlap of the exact evolution with the second-order (n = 2)
    dispersive approximation (Sec. 5.1, Proposition "dispersive differential equation",
    Eq. overlap), without its O(Sigma^5) t term:

        1 - eps - gamma Sigma^3 t,
        eps   = 1 - (share of |g|^2 in the box |k_i - k'_i| <= sigma_i)   (Definition 1),
        gamma = 3 (1 - eps) sum_{|alpha| = 3} |omega^(alpha)_k'| / alpha!,  Sigma = max sigma_i.

    weight: |g(k)|^2 on the wave-vector grid (any normalisation); dk: k - k' on that grid,
    shape weight.shape + (dim,); sigma_box: the box half-widths (dim,); t: scalar or array."""
    w = np.asarray(weight, dtype=float)
    w = w / w.sum()
    sig = np.broadcast_to(np.asarray(sigma_box, dtype=float), (dim,))
    inside = np.all(np.abs(dk) <= sig, axis=-1)
    eps = 1.0 - float(w[inside].sum())
    T = third_derivatives(dim, m, k0)
    acc = 0.0
    for alpha in itertools.product(range(4), repeat=dim):
        if sum(alpha) != 3:
            continue
        idx = tuple(i for i, a in enumerate(alpha) for _ in range(a))
        acc += abs(T[idx]) / float(np.prod([math.factorial(a) for a in alpha]))
    gamma = 3.0 * (1.0 - eps) * acc
    Sigma = float(sig.max())
    return 1.0 - eps - gamma * Sigma ** 3 * np.asarray(t, dtype=float)


def drift_diffusion_overlap(dim, m, k0, weight, dk, omega, t):
    """|<psi~(t)|psi(t)>| for a positive-frequency packet with spectral weights |g(k)|^2: the
    exact phases omega_k against the second-order ones omega' + v.K + K.D.K / 2 (K = dk).
    omega: omega_k on the grid; t: scalar or array."""
    w = np.asarray(weight, dtype=float).ravel()
    w = w / w.sum()
    K = np.asarray(dk, dtype=float).reshape(-1, dim)
    k0 = np.asarray(k0, dtype=float).reshape(dim)
    om0 = float(np.arccos(mass_n(m) * u_derivatives(dim, k0)[0]))
    v, D = drift(dim, m, k0), diffusion(dim, m, k0)
    R = np.asarray(omega, dtype=float).ravel() - (om0 + K @ v + 0.5 * np.einsum("ki,ij,kj->k", K, D, K))
    tt = np.atleast_1d(np.asarray(t, dtype=float))
    out = np.array([abs(np.sum(w * np.exp(-1j * R * x))) for x in tt])
    return out if np.ndim(t) else float(out[0])
