"""qw_step_static (stepping with a static scratch array, no device allocation) against qw_step.

Collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test.  It must pass alone in a fresh process and
after the other tests (the static array keeps whatever an earlier call left).
"""

import numpy as np
import pytest

from paper_1603_06442_gb300 import inputs

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
