"""Extended-precision Fourier evolution for long times.  TEST INFRASTRUCTURE.

psi(t) = U^t psi(0) is reached exactly by the Fourier form of Sec. 4: forward DFT,
the matrix power D_k^t of the symbol per wave vector, inverse DFT.  In FP64 the
eigenphase omega_k t of D_k^t carries about t ulp(omega_k) of rounding in any method
(repeated squaring of D_k included), so at t ~ 1e5 .. 1e7 an FP64 evolution is only
good to ~1e-11 .. 1e-9.  Here D_k^t is taken by repeated squaring of D_k (a library-
free binary power, no closed form) in mpmath at ``dps`` significant digits, with D_k
built from the symbols of Eqs. weyl1d / weyl2d / weyl3d and the Dirac coupling of
Sec. 3.2 at the wave vectors 2 pi j / N evaluated in that precision.  Only the two
DFTs and the final matrix-vector products run in FP64: their rounding (~1e-16) does
not grow with t.  Needs mpmath; used only to write stored expected values on tiny
boxes (tests/golden/make_long_time_spectral.py) and by its own pins.
"""

import mpmath as mp
import numpy as np

from .spectral import dft, idft
from .walk import n_components

__all__ = ["dirac_symbol_mp", "matrix_power_mp", "evolve_mp"]


def _weyl_mp(dim, k):
    """u_k and n~_k (Eqs. weyl1d, weyl2d, weyl3d) at the mp wave vector k (tuple)."""
    if dim == 1:
        return mp.cos(k[0]), (mp.mpf(0), mp.mpf(0), mp.sin(k[0]))
    if dim == 2:
        kx, ky = (k[0] + k[1]) / 2, (k[0] - k[1]) / 2   # lattice wave numbers (k1, k2)
        cx, cy, sx, sy = mp.cos(kx), mp.cos(ky), mp.sin(kx), mp.sin(ky)
        return cx * cy, (sx * cy, cx * sy, sx * sy)
    cx, cy, cz = mp.cos(k[0]), mp.cos(k[1]), mp.cos(k[2])
    sx, sy, sz = mp.sin(k[0]), mp.sin(k[1]), mp.sin(k[2])
    u = cx * cy * cz + sx * sy * sz
    return u, (sx * cy * cz - cx * sy * sz, cx * sy * cz + sx * cy * sz, cx * cy * sz - sx * sy * cz)


def dirac_symbol_mp(dim, m, k):
    """D_k as an mp matrix: 1D [[n e^{-ik}, i m], [i m, n e^{ik}]]; 2D/3D [[n W_k, i m I],
    [i m I, n W_k^dag]] with W_k = u_k I - i sigma . n~_k and n = sqrt(1 - m^2)."""
    m = mp.mpf(m)
    n = mp.sqrt(1 - m * m)
    if dim == 1:
        e = mp.expj(-k[0])
        return mp.matrix([[n * e, 1j * m], [1j * m, n * mp.conj(e)]])
    u, (a, b, c) = _weyl_mp(dim, k)
    # W = u I - i (a sigma_x + b sigma_y + c sigma_z)
    W = [[u - 1j * c, -1j * a - b], [-1j * a + b, u + 1j * c]]
    D = mp.matrix(4, 4)
    for i in range(2):
        for j in range(2):
            D[i, j] = n * W[i][j]
            D[2 + i, 2 + j] = n * mp.conj(W[j][i])
        D[i, 2 + i] = 1j * m
        D[2 + i, i] = 1j * m
    return D


def matrix_power_mp(A, t):
    """A^t by binary powering (repeated squaring) in mp arithmetic."""
    R = mp.eye(A.rows)
    P = A
    t = int(t)
    while t > 0:
        if t & 1:
            R = R * P
        t >>= 1
        if t:
            P = P * P
    return R


def evolve_mp(dim, m, psi, t, dps=50):
    """U^t psi (oracle layout) with D_k^t in `dps`-digit arithmetic at every wave vector of
    the DFT grid (lattice wave numbers in 1D/2D, the Cartesian cube in 3D)."""
    s = n_components(dim)
    psi = np.asarray(psi, dtype=complex)
    N = psi.shape[1]
    ph = dft(psi, dim).reshape(s, -1)
    out = np.empty_like(ph)
    with mp.workdps(dps):
        two_pi_over_N = 2 * mp.pi / N
        for flat, idx in enumerate(np.ndindex(*([N] * dim))):
            k = tuple(two_pi_over_N * j for j in idx)
            Dt = matrix_power_mp(dirac_symbol_mp(dim, m, k), t)
            Dt64 = np.array([[complex(Dt[r, c]) for c in range(s)] for r in range(s)])
            out[:, flat] = Dt64 @ ph[:, flat]
    return idft(out.reshape(psi.shape), dim)
