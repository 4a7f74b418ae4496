"""Pins of the oracle's probability projections (Sec. 5.2: projections of a localised state's
distribution onto axes and planes) against brute force and the walk's light cone.

* brute force: a pure-Python loop over the sites of tiny boxes (every lattice, every keep set);
* localised states project to a delta at the site's coordinates;
* every projection sums to the norm;
* separable fields project to the product's factor;
* light cone: t steps of the update rule (Eq. upd-rule) from a localised state leave exact zeros
  farther than t along any axis (one hop moves every BCC coordinate by 1, the mass term does not
  move), and non-zero probability on the cone's edge.
"""

import itertools

import numpy as np
import pytest

from oracle import walk, observables
from paper_1603_06442_gb300 import inputs


def keep_sets(dim):
    axes = range(dim)
    return [set(c) for r in range(1, dim + 1) for c in itertools.combinations(axes, r)]


def brute(dim, psi, keep):
    N = psi.shape[1]
    kept = sorted(keep)
    out = np.zeros((N,) * len(kept))
    for idx in itertools.product(range(N), repeat=dim):
        d = sum(abs(psi[(s,) + idx]) ** 2 for s in range(psi.shape[0]))
        out[tuple(idx[a] for a in kept)] += d
    return out


def localised(dim, N, site, chi):
    """Normalised state on one lattice site, oracle layout (physical coordinates)."""
    psi = np.zeros((len(chi),) + (N,) * dim, dtype=complex)
    psi[(slice(None),) + tuple(site)] = np.asarray(chi) / np.linalg.norm(chi)
    assert walk.lattice_mask(dim, N)[tuple(site)]
    return psi


@pytest.mark.parametrize("dim,N", [(1, 6), (2, 5), (3, 4), (3, 6)])
def test_projection_brute_force(dim, N):
    psi = walk.from_device(dim, N, inputs.random_field(dim, N, seed=11))
    for keep in keep_sets(dim):
        np.testing.assert_allclose(observables.projection(dim, psi, keep), brute(dim, psi, keep),
                                   rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("dim,N,site", [(1, 12, (5,)), (2, 10, (3, 7)), (3, 8, (2, 4, 6)), (3, 8, (3, 5, 1))])
def test_localised_state_projects_to_a_delta(dim, N, site):
    chi = [1, 0] if dim == 1 else [0.6, 0, 0.8j, 0]
    psi = localised(dim, N, site, chi)
    for keep in keep_sets(dim):
        P = observables.projection(dim, psi, keep)
        at = tuple(site[a] for a in sorted(keep))
        assert abs(P[at] - 1.0) < 1e-14
        assert abs(np.sum(P) - 1.0) < 1e-14


@pytest.mark.parametrize("dim,N", [(1, 64), (2, 24), (3, 16)])
def test_projections_sum_to_the_norm(dim, N):
    psi = 1.3 * walk.from_device(dim, N, inputs.random_field(dim, N, seed=12))
    nrm = observables.norm(psi)
    for keep in keep_sets(dim):
        assert abs(np.sum(observables.projection(dim, psi, keep)) - nrm) <= 1e-12 * nrm


def test_separable_field_projects_to_its_factor():
    N = 12
    rng = np.random.default_rng(5)
    f, g = rng.normal(size=N) + 1j * rng.normal(size=N), rng.normal(size=N) + 1j * rng.normal(size=N)
    chi = np.array([0.5, 0.5j, -0.5, 0.5])
    psi = chi[:, None, None] * f[None, :, None] * g[None, None, :]
    px = observables.projection(2, psi, {0})
    py = observables.projection(2, psi, {1})
    np.testing.assert_allclose(px, np.abs(f) ** 2 * np.sum(np.abs(g) ** 2), rtol=1e-13)
    np.testing.assert_allclose(py, np.abs(g) ** 2 * np.sum(np.abs(f) ** 2), rtol=1e-13)


def torus_dist(a, b, N):
    d = np.abs(a - b) % N
    return np.minimum(d, N - d)


@pytest.mark.parametrize("dim,N,m,t", [(1, 40, 0.3, 9), (2, 24, 0.2, 7), (3, 24, 0.03, 8)])
def test_light_cone_of_a_localised_state(dim, N, m, t):
    site = tuple([N // 2] * dim)
    chi = [1, 0] if dim == 1 else [1, 0, 0, 0]
    psi = walk.step(dim, m, localised(dim, N, site, chi), t)
    for a in range(dim):
        P = observables.projection(dim, psi, {a})
        d = torus_dist(np.arange(N), site[a], N)
        assert np.all(P[d > t] == 0.0)
        assert P[(site[a] + t) % N] > 0 or P[(site[a] - t) % N] > 0
        assert abs(np.sum(P) - 1.0) < 1e-12
