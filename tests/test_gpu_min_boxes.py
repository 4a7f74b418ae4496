"""The smallest boxes of every lattice through the whole API, against the oracle: N = 2 (the
BCC cosets hold one cell each), and odd or factor-3 boxes (1D N=3, 2D N=3, BCC N=6, M = 3).
Plain steps, the Fourier form (Sec. 4), the observables of Sec. 5.2 (norm, <x>, particle
weights), the position moments (Sec. 5.1) and every projection: each kernel's degenerate launch
(a handful of threads, one-cell rows, length-1 or length-3 transforms).

Tolerances as in the other parity tests: relative L2 1e-11 (complex128) / 1e-5 (complex64) for
fields, reductions relative to their scale 1e-12 / 2e-6.
"""

import numpy as np
import pytest

from paper_1603_06442_gb300 import inputs
from oracle import walk, spectral, observables

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

BOXES = [(1, 2), (2, 2), (3, 2), (1, 3), (2, 3), (3, 6)]
FIELD_TOL = {"c128": 1e-11, "c64": 1e-5}
RED_TOL = {"c128": 1e-12, "c64": 2e-6}


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


def field(dim, N, dtype):
    a = inputs.random_field(dim, N, seed=40 + 7 * dim + N)
    npdt = np.complex64 if dtype == "c64" else np.complex128
    return a, walk.from_device(dim, N, a.astype(npdt))


@pytest.mark.parametrize("dim,N", BOXES)
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_min_box_step_and_spectral(qb, dim, N, dtype):
    m = 0.3
    a, psi = field(dim, N, dtype)
    for t in (1, 4):
        plan = qb.Plan(dim, N, m, dtype)
        x = to_dev(a, dtype)
        plan.step(x, t)
        plan.sync()
        got = x.cpu().numpy().astype(np.complex128)
        exp = walk.to_device(dim, N, walk.step(dim, m, psi, t))
        assert rel_l2(got, exp) <= FIELD_TOL[dtype], ("step", t)
        x = to_dev(a, dtype)
        plan.evolve_spectral(x, t)
        plan.sync()
        got = x.cpu().numpy().astype(np.complex128)
        exp = walk.to_device(dim, N, spectral.evolve(dim, m, psi, t))
        assert rel_l2(got, exp) <= FIELD_TOL[dtype], ("spectral", t)
        plan.close()


@pytest.mark.parametrize("dim,N", BOXES)
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_min_box_reductions(qb, dim, N, dtype):
    m = 0.3
    a, psi = field(dim, N, dtype)
    plan = qb.Plan(dim, N, m, dtype)
    x = to_dev(a, dtype)
    tol = RED_TOL[dtype]
    nrm = observables.norm(psi)
    mu = observables.mean_position(dim, psi)
    obs = plan.observables(x)
    assert abs(obs["norm"] - nrm) <= tol * nrm
    for i in range(dim):
        assert abs(obs["x_mean"][i] - mu[i]) <= tol * N
    wp, wm = observables.particle_weights(dim, m, psi)
    assert abs(obs["w_particle"] - wp) <= tol and abs(obs["w_antiparticle"] - wm) <= tol
    mom = plan.position_moments(x)
    cov = observables.position_covariance(dim, psi)
    assert abs(mom["norm"] - nrm) <= tol * nrm
    for i in range(3):
        assert abs(mom["mean"][i] - (mu[i] if i < dim else 0.0)) <= tol * N
        for j in range(3):
            want = cov[i, j] if (i < dim and j < dim) else 0.0
            assert abs(mom["cov"][i][j] - want) <= tol * N * N, (i, j)
    for mask in range(1, 1 << dim):
        axes = {ax for ax in range(dim) if mask >> ax & 1}
        exp = np.transpose(observables.projection(dim, psi, axes))
        got = plan.projection(x, mask).cpu().numpy()
        assert got.shape == exp.shape, mask
        assert np.abs(got - exp).max() <= tol * np.abs(exp).max(), mask
    plan.close()
