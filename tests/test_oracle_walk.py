"""Pins of the oracle's walk definition against what the paper and the mathematics fix.

* Eq. unitarity (Sec. 2): sum_h U_h^dag U_h = sum_h U_h U_h^dag = I and the
  cross sums over equal differences vanish.
* Locality: only the generators of the Cayley graph, their inverses and 0.
* Hand-derived transition tables (tests/golden) from Eqs. weyl2d, weyl3d.
* Dense walk on tiny boxes: unitary, and its spectrum is the multiset
  {exp(-+i omega_k)} with cos omega_k = n u_k (Sec. 3.2) over the DFT grid.
* Special cases: m = 0 in 1D is an exact shift; m = 1 gives D = i*swap; a
  localised state stays inside its light cone (exact zeros); U^dag undoes U.
* The 4-component 1D walk decouples into the 2x2 walk at k and -k (Sec. 3.2).
"""

import os

import numpy as np
import pytest
from scipy.optimize import linear_sum_assignment

from oracle import walk, spectral


def _load_table(path):
    rows = np.loadtxt(path, comments="#")
    out = {}
    d = rows.shape[1] - 8
    for r in rows:
        h = tuple(int(v) for v in r[:d])
        v = r[d:]
        out[h] = np.array([[v[0] + 1j * v[1], v[2] + 1j * v[3]],
                           [v[4] + 1j * v[5], v[6] + 1j * v[7]]]) / 4.0
    return out


@pytest.mark.parametrize("dim", [1, 2, 3])
@pytest.mark.parametrize("m", [0.0, 0.3, 1.0])
def test_transition_unitarity(dim, m):
    mats = walk.transition_matrices(dim, m)
    s = walk.n_components(dim)
    eye = np.eye(s)
    a = sum(U.conj().T @ U for U in mats.values())
    b = sum(U @ U.conj().T for U in mats.values())
    assert np.abs(a - eye).max() < 1e-14
    assert np.abs(b - eye).max() < 1e-14
    keys = list(mats)
    diffs = {tuple(np.subtract(h2, h1)) for h1 in keys for h2 in keys}
    diffs.discard((0,) * dim)
    for d in diffs:
        c1 = sum(mats[h1].conj().T @ mats[h2] for h1 in keys for h2 in keys
                 if tuple(np.subtract(h2, h1)) == d)
        c2 = sum(mats[h2] @ mats[h1].conj().T for h1 in keys for h2 in keys
                 if tuple(np.subtract(h2, h1)) == d)
        assert np.abs(c1).max() < 1e-14, d
        assert np.abs(c2).max() < 1e-14, d


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_locality(dim):
    mats = walk.transition_matrices(dim, 0.4)
    B = walk.lattice_basis(dim)
    gens = [tuple(int(v) for v in b) for b in B]
    if dim == 3:
        gens.append(tuple(int(v) for v in -B.sum(axis=0)))
    expect = set(gens) | {tuple(-v for v in g) for g in gens} | {(0,) * dim}
    assert set(mats) == expect


@pytest.mark.parametrize("dim,fname", [(3, "bcc_weyl_transition.txt"), (2, "square_weyl_transition.txt")])
@pytest.mark.parametrize("m", [0.0, 0.25])
def test_transition_tables_golden(golden_dir, dim, fname, m):
    table = _load_table(os.path.join(golden_dir, fname))
    mats = walk.transition_matrices(dim, m)
    n = walk.mass_n(m)
    assert set(table) == set(mats) - {(0,) * dim}
    for h, W in table.items():
        U = mats[h]
        Wm = table[tuple(-v for v in h)]
        # D_h = diag(n W_h, n (W^dag)_h) with (W^dag)_h = W_{-h}^dag (Sec. 3.2 block form)
        assert np.abs(U[:2, :2] - n * W).max() < 1e-14
        assert np.abs(U[2:, 2:] - n * Wm.conj().T).max() < 1e-14
        assert np.abs(U[:2, 2:]).max() < 1e-14 and np.abs(U[2:, :2]).max() < 1e-14
    U0 = mats.get((0,) * dim, np.zeros((4, 4), dtype=complex))
    expect0 = np.zeros((4, 4), dtype=complex)
    expect0[:2, 2:] = expect0[2:, :2] = 1j * m * np.eye(2)
    assert np.abs(U0 - expect0).max() < 1e-14


def test_transition_1d_explicit():
    m = 0.37
    n = walk.mass_n(m)
    mats = walk.transition_matrices(1, m)
    assert np.abs(mats[(1,)] - np.array([[n, 0], [0, 0]])).max() < 1e-15
    assert np.abs(mats[(-1,)] - np.array([[0, 0], [0, n]])).max() < 1e-15
    assert np.abs(mats[(0,)] - np.array([[0, 1j * m], [1j * m, 0]])).max() < 1e-15


def _match_multisets(a, b):
    cost = np.abs(a[:, None] - b[None, :])
    r, c = linear_sum_assignment(cost)
    return cost[r, c].max()


@pytest.mark.parametrize("dim,N,m", [(1, 8, 0.2), (1, 6, 0.0), (2, 6, 0.3), (2, 4, 0.0),
                                     (3, 4, 0.2), (3, 6, 0.45), (3, 4, 0.0)])
def test_dense_spectrum(dim, N, m):
    U = walk.dense_walk(dim, m, N)
    assert np.abs(U.conj().T @ U - np.eye(U.shape[0])).max() < 1e-13
    ev = np.linalg.eigvals(U)
    k = spectral.k_grid(dim, N).reshape(-1, dim)
    om = walk.dispersion(dim, m, k)
    reps = 1 if dim == 1 else 2
    pred = np.concatenate([np.exp(-1j * om)] * reps + [np.exp(1j * om)] * reps)
    if dim == 3:
        # every BCC wave vector appears 4 times on the cubic grid of the full box
        ev = np.concatenate([ev] * 4)
    assert len(ev) == len(pred)
    assert _match_multisets(ev, pred) < 1e-12


def test_m0_1d_is_shift():
    rng = np.random.default_rng(1)
    N, t = 16, 5
    psi = rng.normal(size=(2, N)) + 1j * rng.normal(size=(2, N))
    out = walk.step(1, 0.0, psi, t)
    assert np.abs(out[0] - np.roll(psi[0], t)).max() < 1e-14
    assert np.abs(out[1] - np.roll(psi[1], -t)).max() < 1e-14


@pytest.mark.parametrize("dim,N", [(1, 8), (2, 6), (3, 4)])
def test_m1_is_i_swap(dim, N):
    rng = np.random.default_rng(2)
    s = walk.n_components(dim)
    psi = rng.normal(size=(s,) + (N,) * dim) + 1j * rng.normal(size=(s,) + (N,) * dim)
    psi *= walk.lattice_mask(dim, N)
    half = s // 2
    for t in range(1, 4):
        out = walk.step(dim, 1.0, psi, t)
        sw = psi if t % 2 == 0 else np.concatenate([psi[half:], psi[:half]])
        assert np.abs(out - (1j ** t) * sw).max() < 1e-14


@pytest.mark.parametrize("dim,N,t", [(1, 32, 9), (2, 24, 7), (3, 20, 5)])
def test_light_cone(dim, N, t):
    s = walk.n_components(dim)
    psi = np.zeros((s,) + (N,) * dim, dtype=complex)
    c = N // 2
    psi[(0,) + (c,) * dim] = 1.0
    out = walk.step(dim, 0.3, psi, t)
    coords = walk.site_coordinates(dim, N)
    if dim == 3:
        hops = np.max([np.abs(x - c) for x in coords], axis=0)       # BCC: (+-1,+-1,+-1) hops
    else:
        hops = np.sum([np.abs(x - c) for x in coords], axis=0)       # axis hops
    dens = np.sum(np.abs(out) ** 2, axis=0)
    assert np.all(dens[hops > t] == 0.0)
    assert dens[hops == t].sum() > 0.0
    assert abs(dens.sum() - 1.0) < 1e-13


@pytest.mark.parametrize("dim,N", [(1, 16), (2, 8), (3, 8)])
def test_adjoint_undoes_step(dim, N):
    rng = np.random.default_rng(3)
    s = walk.n_components(dim)
    psi = (rng.normal(size=(s,) + (N,) * dim) + 1j * rng.normal(size=(s,) + (N,) * dim))
    psi *= walk.lattice_mask(dim, N)
    fwd = walk.step(dim, 0.21, psi, 6)
    back = walk.step(dim, 0.21, fwd, 6, adjoint=True)
    assert np.abs(back - psi).max() < 1e-13


@pytest.mark.parametrize("dim,N", [(1, 64), (2, 16), (3, 12)])
def test_norm_conserved(dim, N):
    rng = np.random.default_rng(4)
    s = walk.n_components(dim)
    psi = (rng.normal(size=(s,) + (N,) * dim) + 1j * rng.normal(size=(s,) + (N,) * dim))
    psi *= walk.lattice_mask(dim, N)
    psi /= np.sqrt(np.sum(np.abs(psi) ** 2))
    out = walk.step(dim, 0.07, psi, 100)
    assert abs(np.sum(np.abs(out) ** 2) - 1.0) < 1e-12


def test_1d_four_component_decouples():
    # D_k of Sec. 3.2 built from the 1D Weyl symbol (Eq. weyl1d) in the 4x4 block form
    m = 0.3
    n = walk.mass_n(m)
    k = np.linspace(-np.pi, np.pi, 17)[:, None]
    W = walk.weyl_matrix(1, k)
    D4 = np.zeros((17, 4, 4), dtype=complex)
    D4[:, :2, :2] = n * W
    D4[:, 2:, 2:] = n * np.conj(np.swapaxes(W, -1, -2))
    D4[:, 0, 2] = D4[:, 1, 3] = D4[:, 2, 0] = D4[:, 3, 1] = 1j * m
    D2p = walk.dirac_symbol(1, m, k)
    D2m = walk.dirac_symbol(1, m, -k)
    assert np.abs(D4[:, [0, 2]][:, :, [0, 2]] - D2p).max() < 1e-15
    assert np.abs(D4[:, [1, 3]][:, :, [1, 3]] - D2m).max() < 1e-15
    assert np.abs(D4[:, [0, 2]][:, :, [1, 3]]).max() < 1e-15


def test_layout_roundtrip():
    rng = np.random.default_rng(5)
    for dim, N, shape in ((1, 8, (2, 8)), (2, 6, (4, 6, 6)), (3, 6, (2, 4, 3, 3, 3))):
        a = rng.normal(size=shape) + 1j * rng.normal(size=shape)
        psi = walk.from_device(dim, N, a)
        assert np.array_equal(walk.to_device(dim, N, psi), a)
        if dim == 3:
            assert np.all(psi[:, ~walk.lattice_mask(3, N)] == 0)
    # device site (coset 1, z=2, y=0, x=1) is the physical site (3, 1, 5)
    a = np.zeros((2, 4, 3, 3, 3), dtype=complex)
    a[1, 2, 2, 0, 1] = 1.0
    psi = walk.from_device(3, 6, a)
    assert psi[2, 3, 1, 5] == 1.0
