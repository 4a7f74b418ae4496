"""Pins of the extended-precision Fourier evolution (oracle/exact.py, Sec. 4).

* At small t it equals the plain update rule applied t times (Eq. upd-rule).
* At moderate t it equals the FP64 Fourier oracle (matrix power of D_k).
* Its binary power of D_k equals the Chebyshev form of the unitary symbol,
  D^t = cos(w t) I + sin(w t)/sin(w) (D - cos(w) I) with cos w = n u_k (Sec. 3.2),
  at t ~ 1e6: two different methods, both in 50 digits.
* Closed forms at t ~ 1e6 where FP64 loses digits: the massless chain is an exact
  shift (U_{+1} = diag(1, 0), U_{-1} = diag(0, 1)) and m = 1 gives D = [[0, i], [i, 0]],
  so psi(t) = i^t swap^t psi(0).
* The norm is conserved at t ~ 1e5.
"""

import numpy as np
import pytest

mp = pytest.importorskip("mpmath")

from oracle import walk, spectral, exact  # noqa: E402
from paper_1603_06442_gb300 import inputs  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dim,N,t", [(1, 16, 7), (2, 6, 5), (3, 4, 3)])
def test_small_t_equals_update_rule(dim, N, t):
    m = 0.27
    psi = walk.from_device(dim, N, inputs.random_field(dim, N, seed=dim))
    assert rel(exact.evolve_mp(dim, m, psi, t, dps=30), walk.step(dim, m, psi, t)) < 1e-13


@pytest.mark.parametrize("dim,N", [(1, 16), (2, 4), (3, 4)])
def test_moderate_t_equals_fp64_fourier_oracle(dim, N):
    m, t = 0.13, 500
    psi = walk.from_device(dim, N, inputs.random_field(dim, N, seed=10 + dim))
    assert rel(exact.evolve_mp(dim, m, psi, t, dps=30), spectral.evolve(dim, m, psi, t)) < 1e-12


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_binary_power_equals_chebyshev_form(dim):
    t = 1000003
    rng = np.random.default_rng(dim)
    with mp.workdps(50):
        for _ in range(3):
            m = mp.mpf(float(rng.uniform(0.01, 0.9)))
            k = tuple(mp.mpf(float(v)) for v in rng.uniform(0, 2 * np.pi, size=dim))
            D = exact.dirac_symbol_mp(dim, m, k)
            s = D.rows
            c = sum(D[i, i] for i in range(s)).real / s        # cos w = n u_k (trace / s)
            w = mp.acos(c)
            cheb = mp.cos(w * t) * mp.eye(s) + (mp.sin(w * t) / mp.sin(w)) * (D - c * mp.eye(s))
            P = exact.matrix_power_mp(D, t)
            assert mp.mnorm(P - cheb, 1) < mp.mpf(10) ** -35


def test_massless_chain_is_an_exact_shift_at_a_million_steps():
    N, t = 16, 1000003
    psi = walk.from_device(1, N, inputs.random_field(1, N, seed=5))
    got = exact.evolve_mp(1, 0.0, psi, t)
    exp = np.stack([np.roll(psi[0], t % N), np.roll(psi[1], -(t % N))])
    assert rel(got, exp) < 1e-14
    # FP64's matrix power drifts by ~t ulp in the phase here
    print("FP64 Fourier oracle at t=%d: rel error %.1e" % (t, rel(spectral.evolve(1, 0.0, psi, t), exp)))


def test_unit_mass_is_a_phase_swap_at_a_million_steps():
    N, t = 8, 1000001
    psi = walk.from_device(2, N, inputs.random_field(2, N, seed=6))
    got = exact.evolve_mp(2, 1.0, psi, t)
    swap = psi[[2, 3, 0, 1]] if t % 2 else psi
    assert rel(got, (1j ** (t % 4)) * swap) < 1e-14


def test_norm_conserved_at_long_times():
    psi = walk.from_device(1, 16, inputs.random_field(1, 16, seed=8))
    got = exact.evolve_mp(1, 0.3, psi, 123457)
    assert abs(np.linalg.norm(got) / np.linalg.norm(psi) - 1) < 1e-14
