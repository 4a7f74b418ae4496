"""GPU parity of qw_projection (probability projections onto axes and planes, Sec. 5.2) against
the oracle, and the localised-state runs of Sec. 5.2 (light cone, projections along axes and
onto the (x, y) plane).

Tolerances, elementwise relative to the largest entry: complex128 1e-13, complex64 2e-6 (site
densities in FP32, sums in FP64).  Light-cone zeros are compared exactly.
"""

import functools

import numpy as np
import pytest

from paper_1603_06442_gb300 import inputs
from oracle import walk, observables

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


def expected(dim, psi, mask):
    """Oracle projection in the device output order (x fastest among the kept axes)."""
    axes = {a for a in range(dim) if mask >> a & 1}
    return np.transpose(observables.projection(dim, psi, axes))


def check(got, exp, dtype, tol=None):
    if tol is None:
        tol = 1e-13 if dtype == "c128" else 2e-6
    scale = float(np.max(np.abs(exp)))
    err = float(np.max(np.abs(got - exp))) / scale
    assert err <= tol, err
    return err


@pytest.mark.parametrize("dim,N", [(1, 64), (1, 1000), (2, 24), (2, 33), (2, 64), (3, 16), (3, 42), (3, 128)])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_projection_matches_oracle(qb, dim, N, dtype):
    a = inputs.random_field(dim, N, seed=90 + N)
    npdt = np.complex64 if dtype == "c64" else np.complex128
    psi = walk.from_device(dim, N, a.astype(npdt))
    plan = qb.Plan(dim, N, 0.2, dtype)
    x = to_dev(a, dtype)
    worst = 0.0
    for mask in range(1, 1 << dim):
        got = plan.projection(x, mask).cpu().numpy()
        assert got.shape == (N,) * bin(mask).count("1")
        worst = max(worst, check(got, expected(dim, psi, mask), dtype))
    plan.close()
    print("projection %dD N=%d %s worst rel err %.2e" % (dim, N, dtype, worst))


def test_projection_is_deterministic(qb):
    dim, N = 3, 64
    x = to_dev(inputs.random_field(dim, N, seed=3), "c64")
    plan = qb.Plan(dim, N, 0.1, "c64")
    for mask in (1, 2, 3, 5, 6):
        a = plan.projection(x, mask).cpu().numpy()
        b = plan.projection(x, mask).cpu().numpy()
        np.testing.assert_array_equal(a, b)
    plan.close()


@functools.lru_cache(maxsize=None)
def localised_run(t):
    dim, N, m = 3, 64, 0.03
    M = N // 2
    a = inputs.localized(dim, N, (0, M // 2, M // 2, M // 2), [1, 0, 0, 0])
    return a, walk.step(dim, m, walk.from_device(dim, N, a), t)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("t", [8, 16, 28])
def test_localised_state_runs(qb, dtype, t):
    """Sec. 5.2: a state on one site with spinor (1, 0, 0, 0), m = 0.03, evolved t steps; its
    projections along y and x and onto the (x, y) plane against the oracle, and exact zeros
    beyond the light cone (t hops along every axis)."""
    dim, N, m = 3, 64, 0.03
    a, psi_t = localised_run(t)
    plan = qb.Plan(dim, N, m, dtype)
    x = to_dev(a, dtype)
    plan.step(x, t)
    plan.sync()
    centre = N // 2
    d = np.abs(np.arange(N) - centre)
    for mask in (5, 6, 3):  # (x, z): along y;  (y, z): along x;  (x, y): onto the plane
        got = plan.projection(x, mask).cpu().numpy()
        # complex64: the t FP32 stencil steps add their own rounding (relative L2 ~1e-6 here)
        check(got, expected(dim, psi_t, mask), dtype, None if dtype == "c128" else 1e-5)
        far = (d[:, None] > t) | (d[None, :] > t)   # either kept coordinate outside the cone
        assert np.all(got[far] == 0.0)
    for mask in (1, 2, 4):
        got = plan.projection(x, mask).cpu().numpy()
        assert np.all(got[d > t] == 0.0)
        assert got[centre + t] > 0 and got[centre - t] > 0
        assert abs(got.sum() - 1.0) < (1e-12 if dtype == "c128" else 1e-5)
    plan.close()


def test_projection_bcc512_sampled(qb):
    """Full-size BCC N=512 (complex64): the (x, y) projection on sampled columns against the
    definition summed on the host in FP64, the x projection against the (x, y) one, both sums
    against the norm."""
    dim, N = 3, 512
    M = N // 2
    a = inputs.gaussian_packet(dim, N, (N / 2,) * 3, 32, [0.3, 0.2, 0.1], [0.5, 0.5j, 0.5, -0.5j])
    host = a.astype(np.complex64)
    plan = qb.Plan(dim, N, 0.1, "c64")
    x = torch.from_numpy(host).cuda()
    pxy = plan.projection(x, 3).cpu().numpy()
    px = plan.projection(x, 1).cpu().numpy()
    nrm = plan.observables(x)["norm"]
    plan.close()
    assert abs(pxy.sum() - nrm) <= 1e-6 * nrm and abs(px.sum() - nrm) <= 1e-6 * nrm
    np.testing.assert_allclose(pxy.sum(axis=0), px, rtol=1e-6, atol=1e-6 * px.max())
    dev = host.reshape(2, 4, M, M, M)
    rng = np.random.default_rng(0)
    for _ in range(64):
        c, my, mx = int(rng.integers(2)), int(rng.integers(M // 4, 3 * M // 4)), int(rng.integers(M // 4, 3 * M // 4))
        col = dev[c, :, :, my, mx].astype(np.complex128)
        exp = float(np.sum(np.abs(col) ** 2))
        X, Y = 2 * mx + c, 2 * my + c
        assert abs(pxy[Y, X] - exp) <= 2e-6 * pxy.max(), (c, my, mx)
        assert pxy[Y, X + 1 if X + 1 < N else X - 1] == 0.0   # mixed parity: not a site


def test_projection_rejects_bad_masks(qb):
    plan = qb.Plan(2, 8, 0.1, "c64")
    x = torch.zeros(plan.elems, dtype=torch.complex64, device="cuda")
    out = torch.empty(64, dtype=torch.float64, device="cuda")
    for mask in (0, 4, 8, -1):
        with pytest.raises(qb.QwError):
            qb.qw_projection(plan.handle, x, mask, out)
    assert qb.qw_projection_elems(plan.handle, 3) == 64
    assert qb.qw_projection_elems(plan.handle, 4) == -1
    plan.close()


def test_misaligned_complex64_projection_matches_aligned(qb):
    """The paired (16-byte) x projection is only used on 16-byte aligned complex64 fields;
    an 8-byte aligned view gets the scalar kernel and the same sums."""
    dim, N = 3, 64
    a = inputs.random_field(dim, N, seed=12).astype(np.complex64)
    plan = qb.Plan(dim, N, 0.1, "c64")
    buf = torch.zeros(a.size + 1, dtype=torch.complex64, device="cuda")
    x_off = buf[1:]
    x_off.copy_(torch.from_numpy(a.ravel()))
    assert x_off.data_ptr() % 16 == 8
    x = torch.from_numpy(a).cuda()
    psi = walk.from_device(dim, N, a.astype(np.complex128))
    for keep in (1, 3, 5, 7):
        p_al = plan.projection(x, keep).cpu().numpy()
        p_off = plan.projection(x_off, keep).cpu().numpy()
        ref = expected(dim, psi, keep)
        scale = np.abs(ref).max()
        assert np.abs(p_off - ref).max() <= 2e-6 * scale, keep
        assert np.abs(p_al - ref).max() <= 2e-6 * scale, keep
    plan.close()


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("N", [64, 42])
def test_bcc_density_writes_every_point(qb, dtype, N):
    """The BCC site density (every axis kept) writes each of the N^3 physical points, the
    zeros of the points that are not sites included, whatever the output held before; an
    8-byte aligned output takes scalar stores and gives the same values."""
    dim = 3
    a = inputs.random_field(dim, N, seed=31 + N)
    npdt = np.complex64 if dtype == "c64" else np.complex128
    psi = walk.from_device(dim, N, a.astype(npdt))
    ref = expected(dim, psi, 7)
    plan = qb.Plan(dim, N, 0.1, dtype)
    x = to_dev(a, dtype)
    n = N ** 3
    buf = torch.full((n + 1,), float("nan"), dtype=torch.float64, device="cuda")
    for out in (buf[:n], buf[1:]):
        out.fill_(float("nan"))
        qb.qw_projection(plan.handle, x, 7, out)
        got = out.cpu().numpy().reshape(ref.shape)
        assert not np.isnan(got).any()
        assert np.all(got[ref == 0] == 0.0)
        check(got, ref, dtype)
    assert buf[1:].data_ptr() % 16 == 8
    plan.close()
