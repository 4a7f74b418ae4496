"""Pins of the oracle's particle-state kinematics (Sec. 5.1, second-order dispersive equation:
drift v = grad omega, diffusion D = grad grad omega) and of its position covariance.

* v and D against central differences of the dispersion omega_k = arccos(n u_k) as the walk
  module computes it (an independent code path), random k, every lattice;
* closed forms: 1D v = n sin k / sin omega; D at k = 0 is (n/m) I in 1D and 3D, (n/2m) I in 2D
  (lattice wave numbers);
* Dirac limit: for small k and m, v -> k / sqrt(m^2 + |k|^2) (Cartesian |k|^2 in 3D);
* exact drift: a positive-frequency packet's mean position moves by t <v>_{|g|^2} (Sec. 5.2:
  the mean of X(0) + V t on the positive part, the Zitterbewegung terms vanish).  On the
  periodic box this holds up to the k-grid sampling of the eigenvector gauge; the boxes are
  taken large enough (BCC N=96, sigma=7: 2.5e-6 sites at t=12; N=64, sigma=5 leaves 1e-3) and
  k0 away from k=0, where the eigenvector formulas are not smooth;
* covariance: brute force on tiny boxes, two-point states, translation invariance.
"""

import itertools

import numpy as np
import pytest

from oracle import walk, observables, kinematics, spectral, states
from paper_1603_06442_gb300 import inputs


def num_grad(f, k, h):
    k = np.asarray(k, dtype=float)
    out = np.zeros(k.size)
    for i in range(k.size):
        e = np.zeros(k.size)
        e[i] = h
        out[i] = (f(k + e) - f(k - e)) / (2 * h)
    return out


@pytest.mark.parametrize("dim", [1, 2, 3])
@pytest.mark.parametrize("m", [0.05, 0.3, 0.8])
def test_drift_and_diffusion_against_differences(dim, m):
    rng = np.random.default_rng(7 + dim)
    om = lambda k: float(walk.dispersion(dim, m, k.reshape(1, dim))[0])
    for _ in range(20):
        k = rng.uniform(-np.pi, np.pi, size=dim)
        v = kinematics.drift(dim, m, k)
        np.testing.assert_allclose(v, num_grad(om, k, 1e-5), atol=2e-8)
        D = kinematics.diffusion(dim, m, k)
        Dn = np.array([num_grad(lambda q: kinematics.drift(dim, m, q)[i], k, 1e-5) for i in range(dim)])
        np.testing.assert_allclose(D, Dn, atol=2e-7)
        np.testing.assert_allclose(D, D.T, atol=1e-14)


@pytest.mark.parametrize("m", [0.1, 0.5])
def test_closed_forms(m):
    n = walk.mass_n(m)
    for k in (0.3, -1.1, 2.5):
        om = np.arccos(n * np.cos(k))
        assert abs(kinematics.drift(1, m, [k])[0] - n * np.sin(k) / np.sin(om)) < 1e-14
    assert abs(kinematics.diffusion(1, m, [0.0])[0, 0] - n / m) < 1e-12
    np.testing.assert_allclose(kinematics.diffusion(3, m, [0, 0, 0]), n / m * np.eye(3), atol=1e-12)
    np.testing.assert_allclose(kinematics.diffusion(2, m, [0, 0]), n / (2 * m) * np.eye(2), atol=1e-12)
    for dim in (1, 2, 3):
        np.testing.assert_allclose(kinematics.drift(dim, m, np.zeros(dim)), 0.0, atol=1e-15)


@pytest.mark.parametrize("dim,order", [(1, 2), (3, 1)])
def test_dirac_limit(dim, order):
    """With k and m scaled by eps, v - k / sqrt(m^2 + |k|^2) is O(eps^2) in 1D and O(eps) on the
    BCC lattice (omega^2 - m^2 - |k|^2 has the cubic term -2 kx ky kz there)."""
    kh = np.array([0.7]) if dim == 1 else np.array([0.4, -0.8, 0.6])
    mh = 0.3
    errs = []
    for eps in (1e-2, 5e-3, 2.5e-3):
        k, m = eps * kh, eps * mh
        v = kinematics.drift(dim, m, k)
        errs.append(np.max(np.abs(v - k / np.sqrt(m * m + k @ k))))
    slopes = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(slopes - order) < 0.1), (errs, slopes)


@pytest.mark.parametrize("dim,N,m,k0,sigma,t", [
    (1, 1024, 0.2, [0.4], 12.0, 150),
    (2, 128, 0.3, [0.5, 0.1], 8.0, 40),
    (3, 96, 0.3, [0.3, 0.2, -0.1], 7.0, 12),
])
def test_positive_packet_drifts_by_the_mean_group_velocity(dim, N, m, k0, sigma, t):
    x0 = [N / 2] * dim
    key = (1, 0) if dim == 1 else (1, 1)
    psi = states.packet(dim, m, N, k0, sigma, x0, {key: 1.0})
    psi_t = spectral.evolve(dim, m, psi, t)
    k = spectral.k_grid(dim, N).reshape(-1, dim)
    dk = states.wrapped_dk(dim, k, np.asarray(k0))
    g2 = np.exp(-2 * sigma * sigma * np.sum(dk * dk, axis=-1))
    vbar = sum(w * kinematics.drift(dim, m, kk) for w, kk in zip(g2, k) if w > 1e-30) / np.sum(g2)
    disp = np.array(observables.mean_position(dim, psi_t)) - np.array(observables.mean_position(dim, psi))
    np.testing.assert_allclose(disp, t * vbar, atol=1e-6 * t)
    # <v> over the packet is the drift at k0 up to the spread of the packet
    assert np.max(np.abs(vbar - kinematics.drift(dim, m, k0))) < 0.05


def brute_cov(dim, psi):
    N = psi.shape[1]
    pts, w = [], []
    for idx in itertools.product(range(N), repeat=dim):
        pts.append(idx)
        w.append(sum(abs(psi[(s,) + idx]) ** 2 for s in range(psi.shape[0])))
    pts, w = np.array(pts, dtype=float), np.array(w)
    mu = (w[:, None] * pts).sum(0) / w.sum()
    d = pts - mu
    return (w[:, None, None] * d[:, :, None] * d[:, None, :]).sum(0) / w.sum()


@pytest.mark.parametrize("dim,N", [(1, 7), (2, 5), (3, 4), (3, 6)])
def test_covariance_brute_force(dim, N):
    psi = walk.from_device(dim, N, inputs.random_field(dim, N, seed=21))
    np.testing.assert_allclose(observables.position_covariance(dim, psi), brute_cov(dim, psi), rtol=1e-12,
                               atol=1e-13)


def test_covariance_two_point_and_translation():
    N = 16
    psi = np.zeros((4, N, N, N), dtype=complex)
    psi[0, 2, 4, 6] = np.sqrt(0.5)
    psi[1, 8, 10, 6] = np.sqrt(0.5)          # both points are BCC sites (all even)
    cov = observables.position_covariance(3, psi)
    d = np.array([6.0, 6.0, 0.0]) / 2
    np.testing.assert_allclose(cov, np.outer(d, d), atol=1e-13)
    shifted = np.roll(psi, (1, 1, 1), axis=(1, 2, 3))   # a lattice translation away from the seam
    np.testing.assert_allclose(observables.position_covariance(3, shifted), cov, atol=1e-12)


def test_positive_packet_spreads_by_the_velocity_spread_1d():
    """1D: the position variance of a positive-frequency packet grows by t^2 Var_{|g|^2}(v) (the
    second moment of X(0) + V t; no interference term), and Var(v) is D(k0)^2 sigma_k^2 to the
    packet's second order (sigma_k^2 = 1/(4 sigma^2) for the amplitude exp(-sigma^2 dk^2))."""
    dim, N, m, k0, sigma = 1, 2048, 0.2, [0.4], 12.0
    psi = states.packet(dim, m, N, k0, sigma, [N / 2], {(1, 0): 1.0})
    k = spectral.k_grid(dim, N).reshape(-1, dim)
    dk = states.wrapped_dk(dim, k, np.asarray(k0))
    g2 = np.exp(-2 * sigma * sigma * np.sum(dk * dk, axis=-1))
    sel = g2 > 1e-30
    w = g2[sel] / g2[sel].sum()
    v = np.array([kinematics.drift(dim, m, kk)[0] for kk in k[sel]])
    var_v = float(np.sum(w * (v - np.sum(w * v)) ** 2))
    c0 = observables.position_covariance(dim, psi)[0, 0]
    for t in (100, 400):
        ct = observables.position_covariance(dim, spectral.evolve(dim, m, psi, t))[0, 0]
        assert abs((ct - c0) - t * t * var_v) <= 1e-6 * t * t * var_v
    D0 = kinematics.diffusion(dim, m, k0)[0, 0]
    assert abs(var_v / (D0 * D0 / (4 * sigma ** 2)) - 1) < 0.15


# ---------------------------------------------------------------- fidelity bound (Eq. overlap)

def test_third_derivatives_against_closed_form_1d():
    """1D: omega = arccos(n cos k); its third derivative by symbolic differentiation."""
    sp = pytest.importorskip("sympy")
    ks, ns = sp.symbols("k n", real=True)
    d3 = sp.lambdify((ks, ns), sp.diff(sp.acos(ns * sp.cos(ks)), ks, 3), "numpy")
    for m in (0.05, 0.3, 0.8):
        n = walk.mass_n(m)
        for k in np.linspace(-2.9, 2.9, 13):
            T = kinematics.third_derivatives(1, m, [k])
            assert abs(T[0, 0, 0] - d3(k, n)) <= 1e-5 * max(1.0, abs(d3(k, n))), (m, k)


@pytest.mark.parametrize("dim", [2, 3])
def test_third_derivatives_against_dispersion_differences(dim):
    """2D/3D: against third-order central differences of the dispersion itself (the walk
    module's arccos(n u_k), a separate code path), every index triple."""
    rng = np.random.default_rng(40 + dim)
    om = lambda k: float(walk.dispersion(dim, 0.3, np.asarray(k).reshape(1, dim))[0])
    h = 2e-3
    for _ in range(4):
        k = rng.uniform(-2.5, 2.5, size=dim)
        T = kinematics.third_derivatives(dim, 0.3, k)
        for i, j, l in itertools.product(range(dim), repeat=3):
            e = np.eye(dim) * h
            f = lambda a, b, c: om(k + a * e[i] + b * e[j] + c * e[l])
            num = sum(sa * sb * sc * f(sa, sb, sc) for sa in (1, -1) for sb in (1, -1) for sc in (1, -1)) / (8 * h ** 3)
            assert abs(T[i, j, l] - num) <= 2e-3 * max(1.0, abs(num)), (dim, i, j, l)


def _particle(dim, N, m, k0, sigma):
    k = spectral.k_grid(dim, N).reshape(-1, dim)
    dk = states.wrapped_dk(dim, k, k0)
    w = np.exp(-2 * sigma * sigma * np.sum(dk * dk, axis=-1))    # |g(k)|^2 of states.packet
    return k, dk, w


@pytest.mark.parametrize("dim,N,m,k0,sigma", [(1, 512, 0.15, [0.3], 12.0), (2, 64, 0.2, [0.4, 0.1], 5.0),
                                              (3, 32, 0.3, [0.2, 0.1, 0.3], 3.0)])
def test_overlap_equals_position_space_overlap(dim, N, m, k0, sigma):
    """The k-space overlap formula against the position-space route: the packet evolved by
    the Fourier oracle (U^t), and the second-order state built as its own DFT with the
    phases omega' + v.K + K.D.K/2, compared by an inner product over the sites."""
    psi0 = states.packet(dim, m, N, k0, sigma, [N / 2] * dim, {(1, 1) if dim > 1 else (1, 0): 1.0})
    k, dk, w = _particle(dim, N, m, k0, sigma)
    om0 = float(walk.dispersion(dim, m, np.asarray(k0).reshape(1, dim))[0])
    v, D = kinematics.drift(dim, m, k0), kinematics.diffusion(dim, m, k0)
    ph2 = om0 + dk @ v + 0.5 * np.einsum("ki,ij,kj->k", dk, D, dk)
    s = walk.n_components(dim)
    for t in (7, 40):
        exact = spectral.evolve(dim, m, psi0, t)
        approx = spectral.idft((spectral.dft(psi0, dim).reshape(s, -1) * np.exp(-1j * ph2 * t)).reshape(psi0.shape),
                               dim)
        pos = abs(np.vdot(approx, exact)) / np.vdot(psi0, psi0).real
        kov = kinematics.drift_diffusion_overlap(dim, m, k0, w, dk, walk.dispersion(dim, m, k), t)
        assert abs(pos - kov) < 1e-10, (t, pos, kov)


def test_overlap_small_t_expansion():
    """1 - |E exp(-i R t)| = t^2 Var(R) / 2 + O(t^4): the overlap's leading decrease is the
    variance of the Taylor remainder R_k of omega beyond second order."""
    dim, N, m, k0, sigma = 1, 2048, 0.1, [0.5], 20.0
    k, dk, w = _particle(dim, N, m, k0, sigma)
    om = walk.dispersion(dim, m, k)
    R = om - (float(walk.dispersion(dim, m, np.array([k0]))[0]) + dk @ kinematics.drift(dim, m, k0)
              + 0.5 * np.einsum("ki,ij,kj->k", dk, kinematics.diffusion(dim, m, k0), dk))
    p = w / w.sum()
    var = float(np.sum(p * R * R) - np.sum(p * R) ** 2)
    for t in (1.0, 3.0, 10.0):
        loss = 1.0 - kinematics.drift_diffusion_overlap(dim, m, k0, w, dk, om, t)
        assert abs(loss - 0.5 * var * t * t) <= 1e-3 * 0.5 * var * t * t, t


@pytest.mark.parametrize("dim,N,m,k0,sigma", [(1, 4096, 0.1, [0.3], 40.0), (1, 4096, 0.6, [1.2], 25.0),
                                              (2, 128, 0.2, [0.4, 0.1], 10.0), (3, 64, 0.3, [0.2, 0.1, 0.3], 6.0)])
def test_overlap_stays_above_the_bound(dim, N, m, k0, sigma):
    """The exact overlap of Eq. overlap is never below the Proposition's bound 1 - eps -
    gamma Sigma^3 t (box half-width 4 standard deviations of |g|^2 per axis), over times
    where the bound is informative; the bound is not vacuous early on."""
    k, dk, w = _particle(dim, N, m, k0, sigma)
    om = walk.dispersion(dim, m, k)
    sb = [4.0 / (2.0 * sigma)] * dim
    t1 = None
    for t in np.linspace(0, 4000, 41):
        b = kinematics.fidelity_bound(dim, m, k0, w, dk, sb, t)
        if b <= 0:
            t1 = t
            break
        o = kinematics.drift_diffusion_overlap(dim, m, k0, w, dk, om, t)
        assert o >= b, (t, o, b)
    assert kinematics.fidelity_bound(dim, m, k0, w, dk, sb, 0.0) > 0.999
    assert t1 is None or t1 > 40
