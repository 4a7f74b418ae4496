"""Pins of the oracle's Fourier evolution and observables.

* numpy FFT against the naive DFT (exact index reduction) and Parseval.
* Spectral evolution (DFT, D_k^t, inverse DFT) equals t updates of the stencil.
* t = 0 is the identity; the 3D result stays on the BCC lattice.
* Chebyshev closed form of D_k^t (cos(omega t) I - i sin(omega t)/sin(omega) G_k,
  from D_k = n u I - i G_k and G_k^2 = sin^2(omega) I) equals the matrix power.
* Particle-weight projector: (I + G_k / sin omega)/2, weights conserved in time
  and equal to |c+|^2 for the paper's eigenvector packets.
"""

import numpy as np
import pytest

from oracle import walk, spectral, observables, states


@pytest.mark.parametrize("N", [1, 2, 3, 5, 8, 12])
def test_fft_matches_naive_dft(N):
    rng = np.random.default_rng(N)
    f = rng.normal(size=(3, N, 4)) + 1j * rng.normal(size=(3, N, 4))
    a = spectral.dft_naive(f, axis=1)
    b = np.fft.fft(f, axis=1)
    assert np.abs(a - b).max() < 1e-12 * max(1, N)
    assert abs(np.sum(np.abs(b) ** 2) / N - np.sum(np.abs(f) ** 2)) < 1e-12 * np.sum(np.abs(f) ** 2)


def test_dft_sign_convention():
    # a plane wave exp(+i k x) lands on the bin of +k under the forward transform
    N = 16
    x = np.arange(N)
    f = np.exp(2j * np.pi * 3 * x / N)[None]
    F = spectral.dft(f, 1)
    assert abs(F[0, 3] - N) < 1e-12 and np.abs(np.delete(F[0], 3)).max() < 1e-12


@pytest.mark.parametrize("dim,N", [(1, 32), (2, 12), (3, 8), (3, 10)])
@pytest.mark.parametrize("t", [0, 1, 7, 20])
def test_spectral_equals_stencil(dim, N, t):
    rng = np.random.default_rng(10 + dim + t)
    s = walk.n_components(dim)
    psi = rng.normal(size=(s,) + (N,) * dim) + 1j * rng.normal(size=(s,) + (N,) * dim)
    psi *= walk.lattice_mask(dim, N)
    m = 0.17
    a = walk.step(dim, m, psi, t)
    b = spectral.evolve(dim, m, psi, t)
    assert np.abs(a - b).max() < 1e-12 * np.abs(psi).max()
    if dim == 3:
        assert np.abs(b[:, ~walk.lattice_mask(3, N)]).max() < 1e-13


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_chebyshev_closed_form(dim):
    rng = np.random.default_rng(20 + dim)
    m = 0.05
    k = rng.uniform(-np.pi, np.pi, size=(64, dim))
    k[0] = 0.0
    D = walk.dirac_symbol(dim, m, k)
    u, nt = walk.weyl_symbol(dim, k)
    n = walk.mass_n(m)
    s = D.shape[-1]
    G = 1j * (D - n * u[:, None, None] * np.eye(s))            # D = n u I - i G
    assert np.abs(G - np.conj(np.swapaxes(G, -1, -2))).max() < 1e-15
    sw = np.sqrt(m * m + n * n * np.sum(nt * nt, axis=-1))   # sin(omega)
    G2 = np.einsum("kij,kjl->kil", G, G)
    assert np.abs(G2 - sw[:, None, None] ** 2 * np.eye(s)).max() < 1e-14
    om = np.arctan2(sw, n * u)
    for t in (1, 2, 17, 1234):
        ratio = np.sin(om * t) / sw
        closed = np.cos(om * t)[:, None, None] * np.eye(s) - 1j * ratio[:, None, None] * G
        assert np.abs(closed - np.linalg.matrix_power(D, t)).max() < 1e-10


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_projector_closed_form(dim):
    rng = np.random.default_rng(30 + dim)
    m = 0.2
    k = rng.uniform(-np.pi, np.pi, size=(32, dim))
    D = walk.dirac_symbol(dim, m, k)
    Pp, Pm = observables.projectors(D)
    u, nt = walk.weyl_symbol(dim, k)
    n = walk.mass_n(m)
    sw = np.sqrt(m * m + n * n * np.sum(nt * nt, axis=-1))
    s = D.shape[-1]
    G = 1j * (D - n * u[:, None, None] * np.eye(s))
    assert np.abs(Pp - 0.5 * (np.eye(s) + G / sw[:, None, None])).max() < 1e-13
    assert np.abs(Pp + Pm - np.eye(s)).max() < 1e-14
    # P+ selects the eigenvalue exp(-i omega)
    om = np.arctan2(sw, n * u)
    DP = np.einsum("kij,kjl->kil", D, Pp)
    assert np.abs(DP - np.exp(-1j * om)[:, None, None] * Pp).max() < 1e-13


@pytest.mark.parametrize("dim,N,m,key_p,key_m", [
    (1, 64, 0.1, (1, 0), (-1, 0)),
    (2, 16, 0.2, (1, 1), (-1, 1)),
    (3, 12, 0.3, (1, -1), (-1, -1)),
])
def test_particle_weights(dim, N, m, key_p, key_m):
    cp, cm = np.sqrt(0.7), np.sqrt(0.3) * np.exp(0.4j)
    psi = states.packet(dim, m, N, [0.3] + [0.1] * (dim - 1), 2.0, [N / 2] * dim,
                        {key_p: cp, key_m: cm})
    wp, wm = observables.particle_weights(dim, m, psi)
    assert abs(wp - 0.7) < 1e-12 and abs(wm - 0.3) < 1e-12
    out = walk.step(dim, m, psi, 9)
    wp2, wm2 = observables.particle_weights(dim, m, out)
    assert abs(wp2 - wp) < 1e-12 and abs(wm2 - wm) < 1e-12
    assert abs(observables.norm(out) - 1.0) < 1e-12


def test_mean_position_simple():
    psi = np.zeros((4, 6, 6, 6), dtype=complex)
    psi[0, 1, 3, 5] = np.sqrt(0.5)
    psi[3, 3, 1, 1] = np.sqrt(0.5)
    assert np.allclose(observables.mean_position(3, psi), [2.0, 2.0, 3.0])
