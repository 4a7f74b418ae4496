"""Physics pins of the oracle: eigenvectors, small-k Dirac limit, Zitterbewegung.

* Eqs. evecs-W / evecs-D: the paper's eigenvector formulas satisfy
  D_k u_{s,p} = exp(-i s omega_k) u_{s,p} and are orthonormal.
* Small-k limit (Eqs. weyl-interpolating, dirac-interp): with k and m scaled by
  eps, omega^2 - (m^2 + |k|^2) = O(eps^4) (O(eps^3) on the BCC lattice) and the interpolating Hamiltonian
  (omega / sin omega) G_k minus the Dirac Hamiltonian is O(eps^2).
* Zitterbewegung (Sec. 5.2, Eqs. meanpos, zitterbewegung, state-zitter): for
  c+ psi+ + c- psi- with |c+| = |c-| the classical drifts cancel and
  <x(t)> - <x(0)> = x_int(t) - x_int(0), x_int(t) = 2 Re[c+* c- sum_k i g^2 e^{2 i omega t}
  <u+|d_k u->] / sum_k g^2.  In 1D, with th(k) = atan2(m, n sin k),
  <u+|d_k u-> = th'/2 and th' = -m n cos k / (m^2 + n^2 sin^2 k), so the jitter
  has frequency 2 omega(k0) and amplitude |c+ c-| m n cos k0 / (m^2 + n^2 sin^2 k0),
  below 1/m as the paper states (Sec. 5.2).
"""

import numpy as np
import pytest
from scipy.optimize import curve_fit

from oracle import walk, spectral, observables, states


@pytest.mark.parametrize("dim", [1, 2, 3])
@pytest.mark.parametrize("m", [0.0, 0.05, 0.3, 0.9])
def test_eigenvectors(dim, m):
    if dim == 1 and m == 0.0:
        pytest.skip("1D eigenvectors are defined for m > 0 (th = atan2(m, .))")
    rng = np.random.default_rng(int(100 * m) + dim)
    k = rng.uniform(-np.pi, np.pi, size=(200, dim))
    k[0] = 0.0
    k[1] = np.pi
    if dim == 3:
        k[2] = [0.0, 0.0, 0.7]          # n~ along z: w = 0
        k[3] = [np.pi / 2, np.pi / 2, 0.0]
    D = walk.dirac_symbol(dim, m, k)
    om = walk.dispersion(dim, m, k)
    ev = states.dirac_eigenvectors(dim, m, k)
    keys = sorted(ev)
    for key in keys:
        s = key[0]
        v = ev[key]
        Dv = np.einsum("kij,kj->ki", D, v)
        assert np.abs(Dv - np.exp(-1j * s * om)[:, None] * v).max() < 1e-12, key
    gram = np.array([[np.sum(np.conj(ev[a]) * ev[b], axis=-1) for b in keys] for a in keys])
    assert np.abs(gram - np.eye(len(keys))[:, :, None]).max() < 1e-12


@pytest.mark.parametrize("dim", [2, 3])
def test_weyl_eigenvectors(dim):
    rng = np.random.default_rng(7)
    k = rng.uniform(-np.pi, np.pi, size=(100, dim))
    W = walk.weyl_matrix(dim, k)
    u, _ = walk.weyl_symbol(dim, k)
    om = np.arccos(u)
    for s, v in states.weyl_eigenvectors(dim, k).items():
        Wv = np.einsum("kij,kj->ki", W, v)
        assert np.abs(Wv - np.exp(-1j * s * om)[:, None] * v).max() < 1e-12


def _physical_k(dim, k):
    if dim == 2:        # Dirac momentum of the square-lattice walk in the (k1 +- k2)/2 reading
        return np.stack([0.5 * (k[..., 0] + k[..., 1]), 0.5 * (k[..., 0] - k[..., 1])], axis=-1)
    return k


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_small_k_dirac_limit(dim):
    rng = np.random.default_rng(40 + dim)
    khat = rng.normal(size=dim)
    mhat = 0.7
    eps = np.array([1e-1, 5e-2, 2.5e-2, 1.25e-2])
    e_disp, e_ham = [], []
    for e in eps:
        m = mhat * e
        k = (khat * e)[None]
        om = walk.dispersion(dim, m, k)[0]
        kp = _physical_k(dim, k)[0]
        e_disp.append(abs(om ** 2 - (m * m + kp @ kp)))
        D = walk.dirac_symbol(dim, m, k)[0]
        u, nt = walk.weyl_symbol(dim, k)
        n = walk.mass_n(m)
        s = D.shape[0]
        G = 1j * (D - n * u[0] * np.eye(s))
        H = om / np.sin(om) * G
        if dim == 1:
            Hd = np.array([[kp[0], -m], [-m, -kp[0]]])
        else:
            sk = np.einsum("j,jab->ab", np.concatenate([kp, np.zeros(3 - len(kp))]), walk.PAULI)
            Hd = np.block([[sk, -m * np.eye(2)], [-m * np.eye(2), -sk]])
        e_ham.append(np.abs(H - Hd).max())
    slope_d = np.polyfit(np.log(eps), np.log(e_disp), 1)[0]
    slope_h = np.polyfit(np.log(eps), np.log(e_ham), 1)[0]
    # 1D/2D: O(eps^4).  BCC: u_k contains s_x s_y s_z, so omega^2 carries the
    # cubic term -2 k_x k_y k_z and the remainder is O(eps^3).
    lo = 2.7 if dim == 3 else 3.7
    assert lo < slope_d < lo + 0.6, slope_d
    assert 1.7 < slope_h < 2.3 if dim > 1 else slope_h > 1.7, slope_h


def test_zitterbewegung_1d():
    """Fig. 5 parameters (m = 0.15, k' = 0.01 pi, c+ = c- = 1/sqrt2) on a wide packet."""
    m, k0, N, sig = 0.15, 0.01 * np.pi, 4096, 200.0
    n = walk.mass_n(m)
    c = 1 / np.sqrt(2)
    x0 = N / 2
    psi = states.packet(1, m, N, [k0], sig, [x0], {(1, 0): c, (-1, 0): c})
    mats = walk.transition_matrices(1, m)
    T = 200
    xs = []
    for _ in range(T + 1):
        xs.append(observables.mean_position(1, psi)[0])
        psi = walk.step(1, m, psi, 1, mats=mats)
    xs = np.array(xs)
    k = 2 * np.pi * np.arange(N) / N
    dk = (k - k0 + np.pi) % (2 * np.pi) - np.pi
    g2 = np.exp(-2 * sig ** 2 * dk ** 2)
    om = np.arccos(n * np.cos(k))
    thp = -m * n * np.cos(k) / (m * m + n * n * np.sin(k) ** 2)
    tt = np.arange(T + 1)
    xint = np.array([2 * np.real(c * c * 1j * np.sum(g2 * np.exp(2j * om * t) * thp / 2)) / np.sum(g2)
                     for t in tt])
    assert np.abs(xs - x0 - xint).max() < 1e-9
    amp = m * n * np.cos(k0) / (2 * (m * m + n * n * np.sin(k0) ** 2))
    freq = 2 * np.arccos(n * np.cos(k0))
    assert amp < 1 / m
    fit, _ = curve_fit(lambda t, a, w, p, b: a * np.cos(w * t + p) + b, tt[:60], xs[:60] - x0,
                       p0=[amp, freq, 0.0, 0.0])
    assert abs(abs(fit[0]) - amp) < 0.01 * amp
    assert abs(fit[1] - freq) < 1e-3 * freq


def test_zitterbewegung_3d():
    """BCC walk, particle + antiparticle packet (u_{+,+} + u_{-,+})/sqrt2 moving along x."""
    m, N, sig = 0.5, 64, 4.0
    k0 = np.array([1.0, 0.0, 0.0])
    x0 = np.array([N / 2] * 3)
    c = 1 / np.sqrt(2)
    psi = states.packet(3, m, N, k0, sig, x0, {(1, 1): c, (-1, 1): c})
    assert np.abs(psi[:, ~walk.lattice_mask(3, N)]).max() < 1e-14
    mats = walk.transition_matrices(3, m)
    T = 14
    xs = []
    for _ in range(T + 1):
        xs.append(observables.mean_position(3, psi))
        psi = walk.step(3, m, psi, 1, mats=mats)
    xs = np.array(xs)
    kg = spectral.k_grid(3, N).reshape(-1, 3)
    dk = states.wrapped_dk(3, kg, k0)
    g2 = np.exp(-2 * sig ** 2 * np.sum(dk * dk, -1))
    om = walk.dispersion(3, m, kg)
    h = 1e-6
    e = np.array([h, 0.0, 0.0])
    up = states.dirac_eigenvectors(3, m, kg)[(1, 1)]
    dum = (states.dirac_eigenvectors(3, m, kg + e)[(-1, 1)]
           - states.dirac_eigenvectors(3, m, kg - e)[(-1, 1)]) / (2 * h)
    d = np.sum(np.conj(up) * dum, -1)
    xint = np.array([2 * np.real(c * c * 1j * np.sum(g2 * np.exp(2j * om * t) * d)) / np.sum(g2)
                     for t in range(T + 1)])
    assert np.ptp(xint) > 0.2
    assert np.abs((xs[:, 0] - xs[0, 0]) - (xint - xint[0])).max() < 5e-5
    # transverse axes: no jitter for this spin, the mean stays put
    assert np.abs(xs[:, 1:] - xs[0, 1:]).max() < 1e-5
