"""GPU parity of qw_position_moments (mean and covariance of the position) against the oracle,
and the particle-state kinematics of Sec. 5.1 on GPU-evolved packets: a positive-frequency
packet drifts by t <v>_{|g|^2} (v = grad omega) and, in 1D, spreads by t^2 Var_{|g|^2}(v).

Tolerances: norm and mean as qw_observables (1e-12 / 1e-6 relative, mean scaled by N);
covariance absolute 1e-12 N^2 (complex128) / 1e-6 N^2 (complex64: FP32 site densities);
kinematics: displacement 1e-6 t sites (complex128) / 2e-4 t (complex64), 1D spread 1e-6 / 1e-3
relative.
"""

import numpy as np
import pytest

from paper_1603_06442_gb300 import inputs
from oracle import walk, observables, kinematics, spectral, states

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def qb(qwlib):
    from paper_1603_06442_gb300 import binding
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return binding


def to_dev(a, dtype):
    npdt = np.complex64 if dtype == "c64" else np.complex128
    return torch.from_numpy(np.ascontiguousarray(a.astype(npdt))).cuda()


def moments_field(dim, N):
    a = inputs.gaussian_packet(dim, N, [N / 3] * dim, N / 9, [0.2] * dim,
                               [1, 0] if dim == 1 else [0.6, 0.8j, 0, 0])
    return a + 0.2 * inputs.random_field(dim, N, 6)


@pytest.mark.parametrize("dim,N", [(1, 64), (1, 999), (1, 1000), (2, 24), (2, 33), (3, 16), (3, 42), (3, 128)])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_position_moments_match_oracle(qb, dim, N, dtype):
    a = moments_field(dim, N)
    plan = qb.Plan(dim, N, 0.1, dtype)
    check_moments(plan, dim, N, dtype, a, to_dev(a, dtype))
    plan.close()


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_position_moments_long_chain(qb, dtype):
    """2^20 sites on one row: far more units than threads, every thread strides over many."""
    dim, N = 1, 1 << 20
    a = moments_field(dim, N)
    plan = qb.Plan(dim, N, 0.1, dtype)
    check_moments(plan, dim, N, dtype, a, to_dev(a, dtype))
    plan.close()


@pytest.mark.parametrize("dim,N", [(1, 1000), (2, 64), (3, 64)])
def test_position_moments_misaligned_complex64(qb, dim, N):
    """Paired (16-byte) loads only on 16-byte aligned complex64 fields: an 8-byte aligned view
    takes the scalar kernel and gives the same moments."""
    a = moments_field(dim, N).astype(np.complex64)
    plan = qb.Plan(dim, N, 0.1, "c64")
    buf = torch.zeros(a.size + 1, dtype=torch.complex64, device="cuda")
    x_off = buf[1:]
    x_off.copy_(torch.from_numpy(a.ravel()))
    assert x_off.data_ptr() % 16 == 8
    check_moments(plan, dim, N, "c64", a, x_off)
    plan.close()


@pytest.mark.parametrize("dim,N", [(1, 4096), (2, 1024), (3, 128)])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_position_covariance_narrow_far_packet(qb, dim, N, dtype):
    """A packet a few sites wide at 0.8 N: its covariance is a small difference of raw moments
    of size (0.8 N)^2, so a coordinate product rounded in the field's precision would show at
    ~1e-7 (0.8 N)^2.  Bound: 2e-5 of the covariance scale in complex64 (FP32 site densities
    alone give ~1e-7), 1e-10 in complex128."""
    a = inputs.gaussian_packet(dim, N, [0.8 * N] * dim, 2.5, [0.3] * dim,
                               [1, 0] if dim == 1 else [0.6, 0.8j, 0, 0])
    npdt = np.complex64 if dtype == "c64" else np.complex128
    psi = walk.from_device(dim, N, a.astype(npdt))
    plan = qb.Plan(dim, N, 0.1, dtype)
    got = plan.position_moments(to_dev(a, dtype))
    plan.close()
    cov = observables.position_covariance(dim, psi)
    scale = float(np.abs(cov).max())
    tol = (2e-5 if dtype == "c64" else 1e-10) * scale
    err = max(abs(got["cov"][i][j] - cov[i, j]) for i in range(dim) for j in range(dim))
    assert err <= tol, (err, scale)


def check_moments(plan, dim, N, dtype, a, x):
    npdt = np.complex64 if dtype == "c64" else np.complex128
    psi = walk.from_device(dim, N, a.astype(npdt))
    got = plan.position_moments(x)
    obs = plan.observables(x)
    rtol = 1e-12 if dtype == "c128" else 1e-6
    ctol = (1e-12 if dtype == "c128" else 1e-6) * N * N
    nrm = observables.norm(psi)
    assert abs(got["norm"] - nrm) <= rtol * nrm
    mu = observables.mean_position(dim, psi)
    cov = observables.position_covariance(dim, psi)
    for i in range(3):
        if i < dim:
            assert abs(got["mean"][i] - mu[i]) <= rtol * N
            assert abs(got["mean"][i] - obs["x_mean"][i]) <= rtol * N
        else:
            assert got["mean"][i] == 0.0
        for j in range(3):
            want = cov[i, j] if (i < dim and j < dim) else 0.0
            assert abs(got["cov"][i][j] - want) <= ctol, (i, j, got["cov"][i][j], want)


def mean_velocity(dim, m, N, k0, sigma):
    k = spectral.k_grid(dim, N).reshape(-1, dim)
    dk = states.wrapped_dk(dim, k, np.asarray(k0))
    g2 = np.exp(-2 * sigma * sigma * np.sum(dk * dk, axis=-1))
    sel = g2 > 1e-30
    w = g2[sel] / g2[sel].sum()
    v = np.array([kinematics.drift(dim, m, kk) for kk in k[sel]])
    vbar = (w[:, None] * v).sum(0)
    cov_v = np.einsum("i,ij,ik->jk", w, v - vbar, v - vbar)
    return vbar, cov_v


DRIFT = [
    (1, 1024, 0.2, [0.4], 12.0, 150),
    (2, 128, 0.3, [0.5, 0.1], 8.0, 40),
    (3, 96, 0.3, [0.3, 0.2, -0.1], 7.0, 12),
]


@pytest.mark.parametrize("dim,N,m,k0,sigma,t", DRIFT)
@pytest.mark.parametrize("dtype,path", [("c128", "spectral"), ("c64", "spectral"), ("c64", "stencil")])
def test_positive_packet_drift_on_gpu(qb, dim, N, m, k0, sigma, t, dtype, path):
    key = (1, 0) if dim == 1 else (1, 1)
    psi0 = states.packet(dim, m, N, k0, sigma, [N / 2] * dim, {key: 1.0})
    vbar, _ = mean_velocity(dim, m, N, k0, sigma)
    plan = qb.Plan(dim, N, m, dtype)
    x = to_dev(walk.to_device(dim, N, psi0), dtype)
    m0 = plan.position_moments(x)
    if path == "spectral":
        plan.evolve_spectral(x, t)
    else:
        plan.step(x, t)
    plan.sync()
    m1 = plan.position_moments(x)
    plan.close()
    disp = np.array(m1["mean"][:dim]) - np.array(m0["mean"][:dim])
    tol = (1e-6 if dtype == "c128" else 2e-4) * t
    np.testing.assert_allclose(disp, t * vbar, atol=tol)
    # and the drift at k0 describes it to the packet's spread
    assert np.max(np.abs(disp / t - kinematics.drift(dim, m, k0))) < 0.05


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_positive_packet_spread_1d_on_gpu(qb, dtype):
    dim, N, m, k0, sigma = 1, 2048, 0.2, [0.4], 12.0
    psi0 = states.packet(dim, m, N, k0, sigma, [N / 2], {(1, 0): 1.0})
    _, cov_v = mean_velocity(dim, m, N, k0, sigma)
    plan = qb.Plan(dim, N, m, dtype)
    x = to_dev(walk.to_device(dim, N, psi0), dtype)
    c0 = plan.position_moments(x)["cov"][0][0]
    rtol = 1e-6 if dtype == "c128" else 1e-3
    t_done = 0
    for t in (100, 400):
        plan.evolve_spectral(x, t - t_done)
        t_done = t
        ct = plan.position_moments(x)["cov"][0][0]
        want = t * t * cov_v[0, 0]
        assert abs((ct - c0) - want) <= rtol * want, (t, ct - c0, want)
    plan.close()


def test_position_moments_rejects_null(qb):
    plan = qb.Plan(1, 8, 0.1, "c64")
    with pytest.raises(qb.QwError):
        qb.qw_position_moments(plan.handle, 0)
    plan.close()


@pytest.mark.parametrize("dim,N,m,k0,sigma,times", [
    (1, 4096, 0.1, [0.3], 40.0, [0, 200, 1000, 3000]),
    (2, 128, 0.2, [0.4, 0.1], 10.0, [0, 50, 150, 300]),
    (3, 64, 0.3, [0.2, 0.1, 0.3], 6.0, [0, 20, 60, 120]),
])
@pytest.mark.parametrize("path", ["spectral_c128", "spectral_c64", "stencil_c64"])
def test_particle_state_overlap_above_fidelity_bound(qb, dim, N, m, k0, sigma, times, path):
    """Sec. 5.1, Proposition "dispersive differential equation", Eq. overlap: a positive-
    frequency particle state evolved on the GPU keeps an overlap with the second-order
    (drift-diffusion) prediction of at least 1 - eps - gamma Sigma^3 t, and that overlap
    equals the oracle's exact one (complex64: 1e-5 absolute; complex128: 1e-10)."""
    method, dtype = path.split("_")
    key = (1, 0) if dim == 1 else (1, 1)
    psi0 = states.packet(dim, m, N, k0, sigma, [N / 2] * dim, {key: 1.0})
    s = walk.n_components(dim)
    k = spectral.k_grid(dim, N).reshape(-1, dim)
    dk = states.wrapped_dk(dim, k, k0)
    w = np.exp(-2 * sigma * sigma * np.sum(dk * dk, axis=-1))   # |g(k)|^2 of states.packet
    om = walk.dispersion(dim, m, k)
    om0 = float(walk.dispersion(dim, m, np.asarray(k0).reshape(1, dim))[0])
    v, D = kinematics.drift(dim, m, k0), kinematics.diffusion(dim, m, k0)
    ph2 = om0 + dk @ v + 0.5 * np.einsum("ki,ij,kj->k", dk, D, dk)
    hat0 = spectral.dft(psi0, dim).reshape(s, -1)
    plan = qb.Plan(dim, N, m, dtype)
    x = to_dev(walk.to_device(dim, N, psi0), dtype)
    done = 0
    worst = 1.0
    for t in times:
        if method == "spectral":
            x = to_dev(walk.to_device(dim, N, psi0), dtype)
            plan.evolve_spectral(x, t)
        else:
            plan.step(x, t - done)
            done = t
        plan.sync()
        got = walk.from_device(dim, N, x.cpu().numpy().astype(np.complex128).reshape(walk.to_device(dim, N, psi0).shape))
        approx = spectral.idft((hat0 * np.exp(-1j * ph2 * t)).reshape(psi0.shape), dim)
        ov = abs(np.vdot(approx, got)) / np.vdot(psi0, psi0).real
        exact = kinematics.drift_diffusion_overlap(dim, m, k0, w, dk, om, t)
        bound = kinematics.fidelity_bound(dim, m, k0, w, dk, [4.0 / (2.0 * sigma)] * dim, t)
        tol = 1e-10 if dtype == "c128" else 1e-5
        print("%s dim=%d t=%d: overlap GPU %.8f oracle %.8f bound %.5f" % (path, dim, t, ov, exact, bound))
        assert abs(ov - exact) <= tol, (t, ov, exact)
        assert ov >= bound - tol, (t, ov, bound)
        worst = min(worst, ov - bound)
    plan.close()
    assert worst >= -1e-5
