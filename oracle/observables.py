"""Observables of a walk state.  TEST INFRASTRUCTURE.

* norm:            sum_x |psi(x)|^2 (unitarity, Eq. un-cond).
* mean position:   <psi|X|psi> / <psi|psi> with X the lattice position operator
                   (Sec. 5.2, X = sum_x x |x><x| (x) I), coordinates in the
                   fixed window [0, N) of the periodic box (lattice coordinates
                   (a, b) in 2D, physical coordinates in 3D).
* second moments:  the covariance of the position over the density,
                   sum (x_i - <x_i>)(x_j - <x_j>) |psi(x)|^2 / norm, same window.
* Foldy-Wouthuysen field (Remark on the Newton-Wigner position): the
                   coefficients phi_r(k) = <u_r(k)|psi^(k)> of the state on the
                   paper's eigenvectors (Eq. evecs-D; 1D: the 2x2 walk's),
                   r = (s, p) in the order (+,+), (+,-), (-,+), (-,-) (1D: +, -),
                   taken back to position space; its mean position is the
                   Newton-Wigner position <X_NW> = <W^-1 psi| X |W^-1 psi>.
* projections:     the probability density sum_s |psi_s(x)|^2 summed over the
                   axes that are not kept (the projections of a localised
                   state's distribution onto axes and planes, Sec. 5.2), on the
                   same window and coordinates as the mean position.
* particle weight: the weight of the positive-frequency part, i.e. of the
                   eigenspace of U_k with eigenvalue exp(-i omega_k) (Eq. eigen-D,
                   s = +).  U_k = cos(omega) I - i G_k with G_k Hermitian, so
                   G_k = i (U_k - U_k^dagger)/2 and the projector is
                   (I + sgn(G_k))/2, sgn taken through a Hermitian eigensolver,
                   with sgn(0) = 0 where omega_k is 0 or pi (both halves share).
"""

import numpy as np

from .walk import site_coordinates
from .spectral import dft, idft, symbol_grid, k_grid
from .states import dirac_eigenvectors

__all__ = ["norm", "mean_position", "position_covariance", "fw_field", "FW_ORDER", "projection", "particle_weights", "projectors"]


def norm(psi):
    """sum |psi|^2 over sites and components."""
    return float(np.sum(np.abs(np.asarray(psi)) ** 2))


def mean_position(dim, psi):
    """<x_i> = sum x_i |psi(x)|^2 / sum |psi(x)|^2, one value per axis."""
    psi = np.asarray(psi)
    N = psi.shape[1]
    dens = np.sum(np.abs(psi) ** 2, axis=0)
    tot = np.sum(dens)
    return [float(np.sum(c * dens) / tot) for c in site_coordinates(dim, N)]


def position_covariance(dim, psi):
    """dim x dim covariance of the position under the normalised density."""
    psi = np.asarray(psi)
    N = psi.shape[1]
    dens = np.sum(np.abs(psi) ** 2, axis=0)
    tot = np.sum(dens)
    xs = site_coordinates(dim, N)
    mu = [np.sum(c * dens) / tot for c in xs]
    cov = np.zeros((dim, dim))
    for i in range(dim):
        for j in range(dim):
            cov[i, j] = np.sum((xs[i] - mu[i]) * (xs[j] - mu[j]) * dens) / tot
    return cov


FW_ORDER = {1: [(1, 0), (-1, 0)], 2: [(1, 1), (1, -1), (-1, 1), (-1, -1)],
            3: [(1, 1), (1, -1), (-1, 1), (-1, -1)]}


def fw_field(dim, m, psi):
    """The state in the eigenbasis of D_k per wave vector, back in position space
    (oracle layout, components in FW_ORDER)."""
    psi = np.asarray(psi, dtype=complex)
    N = psi.shape[1]
    ph = dft(psi, dim)
    ev = dirac_eigenvectors(dim, m, k_grid(dim, N))
    out = np.stack([np.einsum("...i,i...->...", np.conj(ev[key]), ph) for key in FW_ORDER[dim]])
    return idft(out, dim)


def projection(dim, psi, keep):
    """Density summed over the axes not in ``keep`` (a set of axis numbers 0 = x,
    1 = y, 2 = z, each < dim).  Returns an array indexed [x][y][z] over the kept
    axes only, N per axis; on the BCC lattice the physical points that are not
    sites hold 0."""
    psi = np.asarray(psi)
    dens = np.sum(np.abs(psi) ** 2, axis=0)
    drop = tuple(a for a in range(dim) if a not in keep)
    return np.sum(dens, axis=drop) if drop else dens


def projectors(D):
    """(P_plus, P_minus) for stacked unitary symbols D (..., s, s)."""
    G = 0.5j * (D - np.conj(np.swapaxes(D, -1, -2)))
    G = 0.5 * (G + np.conj(np.swapaxes(G, -1, -2)))
    lam, V = np.linalg.eigh(G)
    scale = np.max(np.abs(lam), axis=-1, keepdims=True)
    sgn = np.where(lam > 1e-13, 1.0, np.where(lam < -1e-13, -1.0, 0.0))
    sgn = np.where(scale > 1e-13, sgn, 0.0)
    S = np.einsum("...ij,...j,...kj->...ik", V, sgn, np.conj(V))
    eye = np.eye(D.shape[-1])
    return 0.5 * (eye + S), 0.5 * (eye - S)


def particle_weights(dim, m, psi, chunk=1 << 16):
    """(w_plus, w_minus): weights of the positive / negative frequency parts."""
    psi = np.asarray(psi, dtype=complex)
    s = psi.shape[0]
    N = psi.shape[1]
    ph = dft(psi, dim).reshape(s, -1)
    D = symbol_grid(dim, m, N).reshape(-1, s, s)
    wp = wm = 0.0
    for lo in range(0, D.shape[0], chunk):
        hi = min(lo + chunk, D.shape[0])
        Pp, Pm = projectors(D[lo:hi])
        v = ph[:, lo:hi].T
        wp += float(np.real(np.einsum("ki,kij,kj->", np.conj(v), Pp, v)))
        wm += float(np.real(np.einsum("ki,kij,kj->", np.conj(v), Pm, v)))
    tot = float(np.sum(np.abs(ph) ** 2))
    return wp / tot, wm / tot
