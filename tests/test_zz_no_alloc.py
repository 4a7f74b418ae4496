"""qw_step_static (stepping with a static scratch array, no device allocation) against qw_step.

Collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test.  It must pass alone in a fresh process and
after the other tests (the static array keeps whatever an earlier call left).
"""

import numpy as np
import pytest

from paper_1603_06442_gb300 import inputs
from oracle import walk

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = {"c128": 1e-11, "c64": 1e-5}   # relative L2, as in the other parity tests


@pytest.fixture(scope="module")
def qb(qwlib):
    from paper_1603_06442_gb300 import binding
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return binding


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def to_dev(a, dtype):
    return torch.from_numpy(a.astype(np.complex64 if dtype == "c64" else np.complex128)).cuda()


@pytest.mark.parametrize("dim,N", [(1, 1000), (2, 96), (3, 20), (3, 128)])
@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_static_step_matches_plan_step_twice(qb, dim, N, dtype):
    m = 0.27
    plan = qb.Plan(dim, N, m, dtype)
    for call, (seed, t) in enumerate(((1, 7), (2, 4))):   # two calls in a row
        a = inputs.random_field(dim, N, seed=seed)
        ref = to_dev(a, dtype)
        plan.step(ref, t)
        got = to_dev(a, dtype)
        qb.qw_step_static(dim, N, m, dtype, got, t)
        torch.cuda.synchronize()
        err = rel_l2(got.cpu().numpy(), ref.cpu().numpy())
        assert err <= TOL[dtype], (call, err)
    plan.close()


def test_static_step_rejects_fields_over_the_maximum(qb):
    x = torch.zeros(4, dtype=torch.complex64, device="cuda")
    with pytest.raises(qb.QwError, match="static maximum"):
        qb.qw_step_static(3, 512, 0.1, "c64", x, 1)      # 1 GiB field > 64 MiB
    with pytest.raises(qb.QwError):
        qb.qw_step_static(4, 8, 0.1, "c64", x, 1)


@pytest.mark.parametrize("dim,N,t", [(1, 1000, 9), (2, 40, 6), (3, 20, 5), (3, 128, 3)])
@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_static_step_matches_oracle(qb, dim, N, t, dtype):
    """The allocation-free stepping against the FP64 oracle directly, on two calls in a row
    (the second call starts from the static array's leftovers of the first)."""
    m = 0.19
    a = inputs.random_field(dim, N, seed=N + dim)
    x = to_dev(a, dtype)
    for call in range(2):
        qb.qw_step_static(dim, N, m, dtype, x, t)
        torch.cuda.synchronize()
        exp = walk.to_device(dim, N, walk.step(dim, m, walk.from_device(dim, N, a), t * (call + 1)))
        err = rel_l2(x.cpu().numpy().astype(np.complex128), exp)
        print("qw_step_static vs oracle dim=%d N=%d %s t=%d: rel-L2 %.2e" % (dim, N, dtype, t * (call + 1), err))
        assert err <= TOL[dtype], (call, err)


def test_static_step_misaligned_view(qb):
    """A complex64 field 8 bytes off a 16-byte boundary takes the scalar kernel (the vector
    kernel would need 16-byte alignment) and still matches the oracle."""
    dim, N, m, t = 3, 128, 0.19, 3
    a = inputs.random_field(dim, N, seed=3)
    buf = torch.zeros(a.size + 1, dtype=torch.complex64, device="cuda")
    x = buf[1:]
    x.copy_(torch.from_numpy(a.astype(np.complex64).ravel()))
    assert x.data_ptr() % 16 == 8
    qb.qw_step_static(dim, N, m, "c64", x, t)
    torch.cuda.synchronize()
    exp = walk.to_device(dim, N, walk.step(dim, m, walk.from_device(dim, N, a), t))
    assert rel_l2(x.cpu().numpy().astype(np.complex128).reshape(a.shape), exp) <= TOL["c64"]


def test_static_step_rejects_a_stream_of_another_device(qb):
    """The stream must belong to the current device; only testable with two devices."""
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two CUDA devices")
    x = torch.zeros(2 * 64, dtype=torch.complex64, device="cuda:0")
    with torch.cuda.device(1):
        s1 = torch.cuda.Stream()
    with pytest.raises(qb.QwError, match="stream belongs to device"):
        qb.qw_step_static(1, 64, 0.1, "c64", x, 1, stream=s1)
