"""Pins of the oracle's Foldy-Wouthuysen field and Newton-Wigner position (Remark on the
Newton-Wigner position operator, Eqs. fw, NW, NW-Vt).

* the transform is unitary (norm) and inverted by the eigenvectors (completeness);
* a particle state built on one eigenvector lands in that component only, as the plain
  envelope g, so its Newton-Wigner position is the envelope's centre x0;
* no jitter: for c+ psi+ + c- psi- on one envelope the Newton-Wigner mean moves exactly by
  t (|c+|^2 - |c-|^2) <v> (X_NW(t) = X_NW(0) + V t, null acceleration; the negative-energy
  part moves against v), while the plain mean position jitters (Sec. 5.2).
Boxes are at least 8 packet widths wide, so the seam of the window [0, N) stays below 1e-9.
"""

import numpy as np
import pytest

from oracle import walk, observables, kinematics, spectral, states
from paper_1603_06442_gb300 import inputs


@pytest.mark.parametrize("dim,N", [(1, 32), (2, 12), (3, 8), (3, 12)])
def test_fw_field_is_unitary_and_inverted_by_the_eigenvectors(dim, N):
    m = 0.3
    psi = walk.from_device(dim, N, inputs.random_field(dim, N, seed=31))
    f = observables.fw_field(dim, m, psi)
    assert abs(observables.norm(f) - observables.norm(psi)) < 1e-12
    ev = states.dirac_eigenvectors(dim, m, spectral.k_grid(dim, N))
    fh = spectral.dft(f, dim)
    back = sum(np.moveaxis(ev[key], -1, 0) * fh[r] for r, key in enumerate(observables.FW_ORDER[dim]))
    np.testing.assert_allclose(back, spectral.dft(psi, dim), atol=1e-12)


@pytest.mark.parametrize("dim,N,k0,sigma,key", [
    (1, 256, [0.4], 8.0, (1, 0)),
    (2, 48, [0.5, 0.1], 4.0, (1, -1)),
    (3, 48, [0.3, 0.2, -0.1], 3.0, (-1, 1)),
])
def test_single_eigenvector_packet_is_its_envelope(dim, N, k0, sigma, key):
    m = 0.3
    x0 = [N / 2] * dim
    psi = states.packet(dim, m, N, k0, sigma, x0, {key: 1.0})
    f = observables.fw_field(dim, m, psi)
    r = observables.FW_ORDER[dim].index(key)
    for q in range(f.shape[0]):
        if q != r:
            assert observables.norm(f[q]) < 1e-24
    np.testing.assert_allclose(observables.mean_position(dim, f), x0, atol=1e-9)


def drift_means(dim, m, N, k0, sigma):
    k = spectral.k_grid(dim, N).reshape(-1, dim)
    dk = states.wrapped_dk(dim, k, np.asarray(k0))
    g2 = np.exp(-2 * sigma * sigma * np.sum(dk * dk, axis=-1))
    sel = g2 > 1e-30
    w = g2[sel] / g2[sel].sum()
    return (w[:, None] * np.array([kinematics.drift(dim, m, kk) for kk in k[sel]])).sum(0)


@pytest.mark.parametrize("dim,N,m,k0,sigma,ts,tol", [
    (1, 1024, 0.15, [0.01 * np.pi], 20.0, (5, 17, 40), 1e-9),
    (3, 96, 0.3, [0.0, 0.01 * np.pi, 0.0], 4.0, (3, 7, 11), 1e-8),
])
def test_newton_wigner_position_does_not_jitter(dim, N, m, k0, sigma, ts, tol):
    cp, cm = np.sqrt(0.7), np.sqrt(0.3)
    keys = [(1, 0), (-1, 0)] if dim == 1 else [(1, 1), (-1, 1)]
    x0 = [N / 2] * dim
    psi = states.packet(dim, m, N, k0, sigma, x0, {keys[0]: cp, keys[1]: cm})
    vbar = drift_means(dim, m, N, k0, sigma)
    nw0 = np.array(observables.mean_position(dim, observables.fw_field(dim, m, psi)))
    x_0 = np.array(observables.mean_position(dim, psi))
    jitter = 0.0
    for t in ts:
        pt = spectral.evolve(dim, m, psi, t)
        nw = np.array(observables.mean_position(dim, observables.fw_field(dim, m, pt)))
        np.testing.assert_allclose(nw - nw0, (0.7 - 0.3) * t * vbar, atol=tol)
        jitter = max(jitter, float(np.max(np.abs(np.array(observables.mean_position(dim, pt)) - x_0))))
    assert jitter > 0.05   # the plain mean position does move (Zitterbewegung)
