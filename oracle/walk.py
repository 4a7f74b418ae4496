"""Walk definition: symbols, transition matrices, update rule, layouts.  TEST INFRASTRUCTURE.

Conventions (the readings are listed with their reasons in the design notes):

* Update rule (Sec. 2, Eq. upd-rule with Eq. walk-op):  psi'(x) = sum_h U_h psi(x - h).
  The symbol is U_k = sum_h exp(-i k.h) U_h (Eq. walk-K), so a plane wave
  exp(+i k.x) v is mapped to exp(+i k.x) U_k v.  This is the mirror image of the
  Sec. 2 wording and the form Sec. 5 uses; the dispersion is the same.
* 2D: lattice coordinates (a, b) along h1 = (1,0), h2 = (0,1) (Sec. 3.1).  The
  symbol of Eq. weyl2d is evaluated at k_x = (k1 + k2)/2, k_y = (k1 - k2)/2 with
  k1 = k.h1, k2 = k.h2 (the literal k1 +/- k2 only couples second neighbours).
* 3D: BCC lattice of Eq. bcc-vecs, stored here as a full N^3 periodic cube whose
  sites with x = y = z (mod 2) carry the field and whose other sites stay zero.

Array layouts used by the oracle (complex128):
    dim 1: psi[s, x]          s = 2 components, N sites
    dim 2: psi[s, a, b]       s = 4
    dim 3: psi[s, x, y, z]    s = 4, zero off the BCC lattice
The device layout (components planar, x fastest) is converted by
``from_device`` / ``to_device``.
"""

import numpy as np

__all__ = [
    "mass_n", "n_components", "lattice_basis", "weyl_symbol", "weyl_matrix",
    "dirac_symbol", "k_from_lattice_phases", "transition_matrices", "step",
    "from_device", "to_device", "lattice_mask", "site_coordinates", "dense_walk",
    "dispersion",
]

PAULI = np.array([[[0, 1], [1, 0]], [[0, -1j], [1j, 0]], [[1, 0], [0, -1]]], dtype=complex)


def mass_n(m):
    """n = sqrt(1 - m^2), the Weyl weight of the Dirac coupling (Sec. 3.2, n^2 + m^2 = 1)."""
    m = float(m)
    if not (0.0 <= m <= 1.0):
        raise ValueError("mass must lie in [0, 1]")
    return float(np.sqrt(1.0 - m * m))


def n_components(dim):
    """Coin dimension: 2 in 1D (the 4x4 walk decouples, Sec. 3.2), 4 in 2D and 3D."""
    return 2 if dim == 1 else 4


def lattice_basis(dim):
    """Generators h_j of the Cayley graph (Sec. 3.1, Eq. bcc-vecs); rows are vectors.

    The 3D basis is h1, h2, h3; h4 = -(h1 + h2 + h3) is implied.
    """
    if dim == 1:
        return np.array([[1]])
    if dim == 2:
        return np.array([[1, 0], [0, 1]])
    if dim == 3:
        return np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1]])
    raise ValueError("dim must be 1, 2 or 3")


def weyl_symbol(dim, k):
    """u_k and n~_k of the Weyl walk (Eqs. weyl1d, weyl2d, weyl3d).

    k has shape (..., dim).  dim 1: the wave number; dim 2: the lattice
    wave numbers (k1, k2); dim 3: Cartesian (kx, ky, kz).
    Returns u (...,) and nt (..., 3).
    """
    k = np.asarray(k, dtype=float)
    if dim == 1:
        kk = k[..., 0]
        u = np.cos(kk)
        nt = np.stack([np.zeros_like(kk), np.zeros_like(kk), np.sin(kk)], axis=-1)
        return u, nt
    if dim == 2:
        kx = 0.5 * (k[..., 0] + k[..., 1])
        ky = 0.5 * (k[..., 0] - k[..., 1])
        cx, cy, sx, sy = np.cos(kx), np.cos(ky), np.sin(kx), np.sin(ky)
        u = cx * cy
        nt = np.stack([sx * cy, cx * sy, sx * sy], axis=-1)
        return u, nt
    if dim == 3:
        cx, cy, cz = np.cos(k[..., 0]), np.cos(k[..., 1]), np.cos(k[..., 2])
        sx, sy, sz = np.sin(k[..., 0]), np.sin(k[..., 1]), np.sin(k[..., 2])
        u = cx * cy * cz + sx * sy * sz
        nt = np.stack([sx * cy * cz - cx * sy * sz,
                       cx * sy * cz + sx * cy * sz,
                       cx * cy * sz - sx * sy * cz], axis=-1)
        return u, nt
    raise ValueError("dim must be 1, 2 or 3")


def weyl_matrix(dim, k):
    """W_k = u_k I - i sigma . n~_k (Eq. walk-gen), shape (..., 2, 2)."""
    u, nt = weyl_symbol(dim, k)
    sig = np.einsum("...j,jab->...ab", nt, PAULI)
    eye = np.eye(2, dtype=complex)
    return u[..., None, None] * eye - 1j * sig


def dirac_symbol(dim, m, k):
    """Dirac walk symbol D_k (Sec. 3.2).

    dim 1: the decoupled 2x2 walk [[n e^{-ik}, i m], [i m, n e^{ik}]].
    dim 2, 3: [[n W_k, i m I], [i m I, n W_k^dagger]].
    """
    n = mass_n(m)
    k = np.asarray(k, dtype=float)
    if dim == 1:
        kk = k[..., 0]
        out = np.zeros(kk.shape + (2, 2), dtype=complex)
        out[..., 0, 0] = n * np.exp(-1j * kk)
        out[..., 1, 1] = n * np.exp(1j * kk)
        out[..., 0, 1] = 1j * m
        out[..., 1, 0] = 1j * m
        return out
    W = weyl_matrix(dim, k)
    Wd = np.conj(np.swapaxes(W, -1, -2))
    out = np.zeros(W.shape[:-2] + (4, 4), dtype=complex)
    out[..., :2, :2] = n * W
    out[..., 2:, 2:] = n * Wd
    out[..., 0, 2] = out[..., 1, 3] = 1j * m
    out[..., 2, 0] = out[..., 3, 1] = 1j * m
    return out


def dispersion(dim, m, k):
    """omega_k = arccos(n u_k) (Sec. 3.2; for dim 1, n cos k)."""
    u, _ = weyl_symbol(dim, k)
    return np.arccos(np.clip(mass_n(m) * u, -1.0, 1.0))


def k_from_lattice_phases(dim, theta):
    """Wave vector k with k . h_j = theta_j for the basis of ``lattice_basis``."""
    B = lattice_basis(dim).astype(float)
    theta = np.asarray(theta, dtype=float)
    return np.linalg.solve(B, theta.reshape(-1, dim).T).T.reshape(theta.shape)


def transition_matrices(dim, m, grid=16, tol=1e-12):
    """Position-space transition matrices U_h as Fourier coefficients of D_k.

    From Eq. walk-K, D_k = sum_h exp(-i k.h) U_h.  Writing h = sum_j a_j h_j and
    theta_j = k.h_j, the coefficient of the integer vector a is
    (1/G^d) sum_theta D(theta) exp(+i a.theta) on a G^d grid of theta.
    Returns {h (tuple, Cartesian / lattice coordinates): U_h (s x s)} for all
    coefficients above ``tol``.
    """
    th1 = 2.0 * np.pi * np.arange(grid) / grid
    mesh = np.meshgrid(*([th1] * dim), indexing="ij")
    theta = np.stack(mesh, axis=-1)
    k = k_from_lattice_phases(dim, theta)
    D = dirac_symbol(dim, m, k)
    coef = np.fft.ifftn(D, axes=tuple(range(dim)))
    B = lattice_basis(dim)
    out = {}
    for idx in np.ndindex(*([grid] * dim)):
        C = coef[idx]
        if np.max(np.abs(C)) <= tol:
            continue
        a = np.array([i if i <= grid // 2 else i - grid for i in idx])
        h = tuple(int(v) for v in a @ B)
        out[h] = C
    return out


def _roll(psi, h):
    """(T psi)(x) = psi(x - h) on the periodic box: np.roll by +h on the spatial axes."""
    return np.roll(psi, shift=tuple(h), axis=tuple(range(1, 1 + len(h))))


def step(dim, m, psi, nsteps=1, adjoint=False, mats=None):
    """Apply the update rule psi'(x) = sum_h U_h psi(x - h)  (Eq. upd-rule), nsteps times.

    adjoint=True applies U^dagger: psi'(x) = sum_h U_h^dagger psi(x + h).
    Generic complex matrix-vector products over every transition matrix.
    """
    if mats is None:
        mats = transition_matrices(dim, m)
    psi = np.array(psi, dtype=complex, copy=True)
    for _ in range(int(nsteps)):
        new = np.zeros_like(psi)
        for h, U in mats.items():
            if adjoint:
                new += np.einsum("rs,s...->r...", np.conj(U.T), _roll(psi, tuple(-v for v in h)))
            else:
                new += np.einsum("rs,s...->r...", U, _roll(psi, h))
        psi = new
    return psi


def lattice_mask(dim, N):
    """Boolean mask of lattice sites in the oracle layout (all sites in 1D/2D; BCC in 3D)."""
    if dim in (1, 2):
        return np.ones((N,) * dim, dtype=bool)
    x, y, z = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    return ((x - y) % 2 == 0) & ((y - z) % 2 == 0)


def site_coordinates(dim, N):
    """Coordinate arrays (one per axis) in [0, N), oracle layout."""
    return np.meshgrid(*([np.arange(N)] * dim), indexing="ij")


def from_device(dim, N, arr):
    """Device layout -> oracle layout.

    Device: dim 1 [s][x]; dim 2 [s][y][x]; dim 3 [coset][s][z][y][x] with
    coset c holding the physical site 2*(mx, my, mz) + c*(1, 1, 1), M = N/2.
    """
    arr = np.asarray(arr)
    if dim == 1:
        return np.array(arr.reshape(2, N), dtype=complex)
    if dim == 2:
        return np.array(arr.reshape(4, N, N).transpose(0, 2, 1), dtype=complex)
    M = N // 2
    a = arr.reshape(2, 4, M, M, M)
    psi = np.zeros((4, N, N, N), dtype=complex)
    for c in (0, 1):
        psi[:, c::2, c::2, c::2] = a[c].transpose(0, 3, 2, 1)
    return psi


def to_device(dim, N, psi):
    """Oracle layout -> device layout (inverse of ``from_device``), complex128."""
    psi = np.asarray(psi, dtype=complex)
    if dim == 1:
        return psi.copy()
    if dim == 2:
        return np.ascontiguousarray(psi.transpose(0, 2, 1))
    M = N // 2
    out = np.zeros((2, 4, M, M, M), dtype=complex)
    for c in (0, 1):
        out[c] = psi[:, c::2, c::2, c::2].transpose(0, 3, 2, 1)
    return out


def dense_walk(dim, m, N):
    """The full walk unitary on the periodic box, one column per basis state.

    Only lattice sites are kept (BCC sites in 3D); size (s*|V|)^2.  Small N only.
    """
    s = n_components(dim)
    mask = lattice_mask(dim, N)
    idx = np.argwhere(mask)
    mats = transition_matrices(dim, m)
    cols = []
    for site in idx:
        for comp in range(s):
            e = np.zeros((s,) + (N,) * dim, dtype=complex)
            e[(comp,) + tuple(site)] = 1.0
            out = step(dim, m, e, 1, mats=mats)
            cols.append(out[(slice(None),) + tuple(idx.T)].T.reshape(-1))
    return np.array(cols).T
