"""Eigenvectors and particle-state packets.  TEST INFRASTRUCTURE.

* Weyl eigenvectors (Eq. evecs-W): with W_k = [[z, -w*], [w, z*]],
  Re z = u_k, n~_k = (-Im w, Re w, -Im z),
  u^W_s = (1/sqrt2) (sqrt(1 - s v^W), -s e^{i phi} sqrt(1 + s v^W)),
  v^W = Im z / sqrt(1 - u^2), phi = Arg w - pi/2.
* Dirac eigenvectors (Eq. evecs-D), s = energy sign (eigenvalue exp(-i s omega)),
  p = spin, v^D = n sqrt(1 - u^2) / sqrt(1 - n^2 u^2).
  Where n~_k = 0 both ratios are 0/0; there v^W = 0 and phi = 0 are taken (and
  v^D = 0 when also m = 0), which still gives an orthonormal eigenbasis.
* 1D (the decoupled 2x2 walk of Sec. 3.2): G_k = n sin k sigma_z - m sigma_x, so
  G_k / sin(omega) = cos(th) sigma_z - sin(th) sigma_x with th = atan2(m, n sin k),
  whose eigenvectors are u_+ = (cos th/2, -sin th/2), u_- = (sin th/2, cos th/2).
* Particle-state packet (Definition 1, Eq. state-zitter): psi^(k) = g(k) sum c u(k),
  g(k) = exp(-sigma^2 |dk|^2) exp(-i k.x0), dk = k - k0 reduced per lattice
  direction into (-pi, pi]; sigma is the spatial width in sites.
"""

import numpy as np

from .walk import mass_n, weyl_symbol, n_components, lattice_basis, k_from_lattice_phases
from .spectral import k_grid, idft

__all__ = ["weyl_eigenvectors", "dirac_eigenvectors", "packet", "wrapped_dk"]

_TINY = 1e-12


def _weyl_parts(dim, k):
    u, nt = weyl_symbol(dim, k)
    z = u - 1j * nt[..., 2]
    w = nt[..., 1] - 1j * nt[..., 0]
    # sqrt(1 - u^2) = |n~| because u^2 + |n~|^2 = 1 (W_k unitary); the second
    # form keeps its digits where u^2 is close to 1.
    r = np.sqrt(np.sum(nt * nt, axis=-1))
    small = r < _TINY
    vW = np.where(small, 0.0, np.imag(z) / np.where(small, 1.0, r))
    vW = np.clip(vW, -1.0, 1.0)
    # Arg w is undefined where w = 0 (n~ along z): any phase gives an
    # eigenvector there; phi = 0 is taken (also below rounding level, so that
    # wave vectors equal modulo the reciprocal lattice get equal vectors).
    phi = np.where(np.abs(w) > _TINY, np.angle(w) - 0.5 * np.pi, 0.0)
    return u, vW, phi, r


def weyl_eigenvectors(dim, k):
    """{s: u^W_s(k)} for s = +1, -1, each shape (..., 2)  (Eq. evecs-W; dim 2, 3)."""
    u, vW, phi, _ = _weyl_parts(dim, k)
    out = {}
    for s in (1, -1):
        e = np.stack([np.sqrt(1 - s * vW) + 0j,
                      -s * np.exp(1j * phi) * np.sqrt(1 + s * vW)], axis=-1)
        out[s] = e / np.sqrt(2.0)
    return out


def dirac_eigenvectors(dim, m, k):
    """{(s, p): u^D_{s,p}(k)} with D_k u = exp(-i s omega_k) u.

    dim 2, 3: Eq. evecs-D, shape (..., 4).  dim 1: {(s, 0)} of the 2x2 walk.
    """
    n = mass_n(m)
    k = np.asarray(k, dtype=float)
    if dim == 1:
        th = np.arctan2(m, n * np.sin(k[..., 0]))
        c, sn = np.cos(0.5 * th), np.sin(0.5 * th)
        return {(1, 0): np.stack([c, -sn], axis=-1) + 0j,
                (-1, 0): np.stack([sn, c], axis=-1) + 0j}
    u, vW, phi, r = _weyl_parts(dim, k)
    # sqrt(1 - n^2 u^2) = sqrt(m^2 + n^2 |n~|^2) by the same identity.
    den = np.sqrt(m * m + n * n * r * r)
    vD = np.where(den > _TINY, n * r / np.where(den > _TINY, den, 1.0), 0.0)
    vD = np.clip(vD, -1.0, 1.0)
    ep = np.exp(1j * phi)
    out = {}
    for s in (1, -1):
        for p in (1, -1):
            e = np.stack([
                np.sqrt((1 - p * vW) * (1 + s * p * vD)) + 0j,
                -p * ep * np.sqrt((1 + p * vW) * (1 + s * p * vD)),
                -s * np.sqrt((1 - p * vW) * (1 - s * p * vD)) + 0j,
                s * p * ep * np.sqrt((1 + p * vW) * (1 - s * p * vD)),
            ], axis=-1)
            out[(s, p)] = 0.5 * e
    return out


def wrapped_dk(dim, k, k0):
    """k - k0 reduced into (-pi, pi] along each lattice direction, returned as a wave vector."""
    B = lattice_basis(dim).astype(float)
    d = np.asarray(k, dtype=float) - np.asarray(k0, dtype=float)
    th = d @ B.T
    th = th - 2.0 * np.pi * np.round(th / (2.0 * np.pi))
    return k_from_lattice_phases(dim, th)


def packet(dim, m, N, k0, sigma, x0, coeffs):
    """Normalised particle-state packet on the periodic box (oracle layout).

    coeffs: {(s, p): c} over the keys of ``dirac_eigenvectors``.
    """
    k = k_grid(dim, N)
    dk = wrapped_dk(dim, k, k0)
    x0 = np.asarray(x0, dtype=float).reshape(dim)
    g = np.exp(-sigma * sigma * np.sum(dk * dk, axis=-1)) * np.exp(-1j * (k @ x0))
    ev = dirac_eigenvectors(dim, m, k)
    spin = sum(c * ev[key] for key, c in coeffs.items())
    ph = np.moveaxis(g[..., None] * spin, -1, 0)
    psi = idft(ph, dim)
    s = n_components(dim)
    assert psi.shape[0] == s
    return psi / np.sqrt(np.sum(np.abs(psi) ** 2))
