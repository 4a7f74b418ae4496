"""GPU parity of qw_fw_transform (Foldy-Wouthuysen field; the Remark on the Newton-Wigner
position) against the oracle, and the jitter-free Newton-Wigner mean of particle-antiparticle
packets evolved on the GPU.

Tolerances: relative L2 of the field 1e-11 (complex128) / 1e-5 (complex64); Newton-Wigner
displacement against (|c+|^2 - |c-|^2) t <v>: 1e-8 sites (complex128) / 2e-4 t (complex64).
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


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dim,N", [(1, 64), (1, 1024), (2, 24), (2, 64), (3, 16), (3, 36), (3, 128)])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_fw_field_matches_oracle(qb, dim, N, dtype):
    m = 0.3
    a = inputs.random_field(dim, N, seed=50 + N)
    npdt = np.complex64 if dtype == "c64" else np.complex128
    psi = walk.from_device(dim, N, a.astype(npdt))
    plan = qb.Plan(dim, N, m, dtype)
    x = to_dev(a, dtype)
    f = plan.fw_transform(x)
    got = walk.from_device(dim, N, f.cpu().numpy().astype(np.complex128))
    plan.close()
    err = rel_l2(got, observables.fw_field(dim, m, psi))
    print("FW field %dD N=%d %s rel-L2 %.2e" % (dim, N, dtype, err))
    assert err <= (1e-11 if dtype == "c128" else 1e-5), err
    # the input is left as it was
    np.testing.assert_array_equal(x.cpu().numpy(), a.astype(npdt))


def test_fw_transform_in_place(qb):
    dim, N, m = 3, 32, 0.2
    a = inputs.random_field(dim, N, seed=4).astype(np.complex64)
    plan = qb.Plan(dim, N, m, "c64")
    x = to_dev(a, "c64")
    ref = plan.fw_transform(x).cpu().numpy()
    plan.fw_transform(x, out=x)
    np.testing.assert_allclose(x.cpu().numpy(), ref, rtol=0, atol=1e-6)
    plan.close()


def mean_drift(dim, m, N, k0, sigma):
    k = spectral.k_grid(dim, N).reshape(-1, dim)
    dk = states.wrapped_dk(dim, k, np.asarray(k0))
    g2 = np.exp(-2 * sigma * sigma * np.sum(dk * dk, axis=-1))
    sel = g2 > 1e-30
    w = g2[sel] / g2[sel].sum()
    return (w[:, None] * np.array([kinematics.drift(dim, m, kk) for kk in k[sel]])).sum(0)


@pytest.mark.parametrize("dim,N,m,k0,sigma,ts", [
    (1, 1024, 0.15, [0.01 * np.pi], 20.0, (5, 17, 40)),
    (3, 96, 0.3, [0.0, 0.01 * np.pi, 0.0], 4.0, (3, 7, 11)),
])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_newton_wigner_mean_does_not_jitter_on_gpu(qb, dim, N, m, k0, sigma, ts, dtype):
    keys = [(1, 0), (-1, 0)] if dim == 1 else [(1, 1), (-1, 1)]
    psi0 = states.packet(dim, m, N, k0, sigma, [N / 2] * dim, {keys[0]: np.sqrt(0.7), keys[1]: np.sqrt(0.3)})
    vbar = mean_drift(dim, m, N, k0, sigma)
    plan = qb.Plan(dim, N, m, dtype)
    x = to_dev(walk.to_device(dim, N, psi0), dtype)
    f = torch.empty_like(x)
    plan.fw_transform(x, out=f)
    nw0 = np.array(plan.position_moments(f)["mean"][:dim])
    x_0 = np.array(plan.position_moments(x)["mean"][:dim])
    jitter, done = 0.0, 0
    for t in ts:
        plan.evolve_spectral(x, t - done)
        done = t
        plan.fw_transform(x, out=f)
        nw = np.array(plan.position_moments(f)["mean"][:dim])
        tol = 1e-8 if dtype == "c128" else 2e-4 * t
        np.testing.assert_allclose(nw - nw0, 0.4 * t * vbar, atol=tol)
        xm = np.array(plan.position_moments(x)["mean"][:dim])
        jitter = max(jitter, float(np.max(np.abs(xm - x_0))))
    plan.close()
    assert jitter > 0.05


def test_fw_transform_needs_spectral_sizes(qb):
    plan = qb.Plan(2, 14, 0.1, "c64")      # 14 is not 2^a 3^b
    x = torch.zeros(plan.elems, dtype=torch.complex64, device="cuda")
    with pytest.raises(qb.QwError):
        plan.fw_transform(x)
    plan.close()
