"""Fourier evolution psi(t) = U^t psi(0) through the DFT (Sec. 4).  TEST INFRASTRUCTURE.

The Fourier form reaches exactly the result of t updates, so the oracle writes
the plain definition out: forward DFT (sum_x psi(x) exp(-i k.x)), multiply each
wave vector by the matrix power D_k^t of the symbol (repeated squaring, a
library primitive, no closed form), inverse DFT (1/|V| sum_k ... exp(+i k.x)).

In 3D the field lives on the full N^3 cube (zero off the BCC lattice), so the
plain cubic DFT is used; each BCC wave vector then appears four times (k and
k + reciprocal FCC vectors) with equal values, and D_k is periodic under those
shifts, so the inverse transform stays on the lattice.  The paper's two-coset
reduction (Eqs. bcc-dft, bcc-idft) is not used here: it is what the CUDA path
does, and this oracle checks it.
"""

import numpy as np

from .walk import dirac_symbol, n_components

__all__ = ["dft_naive", "dft", "idft", "k_grid", "evolve", "symbol_grid"]


def dft_naive(f, axis):
    """Naive forward DFT along one axis: F[k] = sum_x f[x] exp(-2 pi i k x / N).

    Twiddles are read from a cos/sin table at the exact index (k*x) mod N.
    """
    f = np.moveaxis(np.asarray(f, dtype=complex), axis, 0)
    N = f.shape[0]
    ang = 2.0 * np.pi * np.arange(N) / N
    table = np.cos(ang) - 1j * np.sin(ang)
    out = np.zeros_like(f)
    for k in range(N):
        for x in range(N):
            out[k] += table[(k * x) % N] * f[x]
    return np.moveaxis(out, 0, axis)


def dft(psi, dim):
    """Forward DFT over the spatial axes 1..dim (numpy FFT, exp(-i k.x), unnormalised)."""
    return np.fft.fftn(psi, axes=tuple(range(1, dim + 1)))


def idft(psi_hat, dim):
    """Inverse DFT over the spatial axes, 1/|V| normalisation, exp(+i k.x)."""
    return np.fft.ifftn(psi_hat, axes=tuple(range(1, dim + 1)))


def k_grid(dim, N):
    """Wave vectors 2 pi j / N of the DFT grid in the oracle layout, shape (N,)*dim + (dim,).

    dim 1, 2: lattice wave numbers; dim 3: Cartesian wave vector of the cube.
    """
    k1 = 2.0 * np.pi * np.arange(N) / N
    return np.stack(np.meshgrid(*([k1] * dim), indexing="ij"), axis=-1)


def symbol_grid(dim, m, N):
    """D_k on the DFT grid, shape (N,)*dim + (s, s)."""
    return dirac_symbol(dim, m, k_grid(dim, N))


def evolve(dim, m, psi, t, chunk=1 << 16):
    """U^t psi via DFT -> D_k^t (matrix power) -> inverse DFT."""
    t = int(t)
    if t < 0:
        raise ValueError("t must be >= 0")
    s = n_components(dim)
    psi = np.asarray(psi, dtype=complex)
    N = psi.shape[1]
    ph = dft(psi, dim).reshape(s, -1)
    k = k_grid(dim, N).reshape(-1, dim)
    out = np.empty_like(ph)
    for lo in range(0, k.shape[0], chunk):
        hi = min(lo + chunk, k.shape[0])
        D = dirac_symbol(dim, m, k[lo:hi])
        Dt = np.linalg.matrix_power(D, t)
        out[:, lo:hi] = np.einsum("krs,sk->rk", Dt, ph[:, lo:hi])
    return idft(out.reshape(psi.shape), dim)
