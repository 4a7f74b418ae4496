"""Debug poison (qw_set_debug_poison): scratch and partner buffers filled with NaN before every
call that must write them before reading them.  Every stencil variant, the observables, the
allocation-free stepping and a batch captured while poison is on still match the oracle, so no
kernel reads memory it did not write first."""

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
    binding.qw_set_debug_poison(True)
    yield binding
    binding.qw_set_debug_poison(False)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


# box sides whose axis lengths are 2^a 3^b, so that the observables' particle weights (through
# the forward DFT in the plan's scratch field) run under poison too
@pytest.mark.parametrize("dim,N,variant", [(1, 324, "plain"), (1, 324, "fused"), (2, 48, "plain"), (2, 48, "fused"),
                                           (3, 24, "plain"), (3, 128, "vec"), (3, 128, "tma"), (3, 128, "tma2"),
                                           (3, 24, "fused")])
def test_stencil_variants_under_poison(qb, dim, N, variant):
    m, t = 0.21, 7
    a = inputs.random_field(dim, N, seed=31 + dim)
    plan = qb.Plan(dim, N, m, "c64")
    plan.set_stencil(variant)
    x = torch.from_numpy(a.astype(np.complex64)).cuda()
    plan.step(x, t)
    obs = plan.observables(x)
    plan.sync()
    got = x.cpu().numpy().astype(np.complex128)
    plan.close()
    assert np.all(np.isfinite(got))
    exp = walk.to_device(dim, N, walk.step(dim, m, walk.from_device(dim, N, a), t))
    assert rel_l2(got, exp) <= 1e-5
    psi = walk.from_device(dim, N, exp)
    assert abs(obs["norm"] - observables.norm(psi)) < 1e-4 and np.isfinite(obs["w_particle"])


def test_static_step_and_batch_under_poison(qb):
    a = inputs.random_field(2, 48, seed=3)
    x = torch.from_numpy(a.astype(np.complex64)).cuda()
    qb.qw_step_static(2, 48, 0.3, "c64", x, 5)
    torch.cuda.synchronize()
    exp = walk.to_device(2, 48, walk.step(2, 0.3, walk.from_device(2, 48, a), 5))
    assert rel_l2(x.cpu().numpy(), exp) <= 1e-5
    spec = [(2, 40, 0.2, 9), (3, 16, 0.3, 6), (1, 200, 0.1, 7)]
    fields = [inputs.random_field(d, N, seed=50 + i) for i, (d, N, m, t) in enumerate(spec)]
    dev = [torch.from_numpy(f.astype(np.complex64)).cuda() for f in fields]
    b = qb.Batch([(d, N, m, t, xx) for (d, N, m, t), xx in zip(spec, dev)])
    for depth in (1, 2):
        for f, xx in zip(fields, dev):
            xx.copy_(torch.from_numpy(f.astype(np.complex64)))
        b.set_tiling({"tile_sites": 512, "l2_budget_bytes": 16 << 30, "depth": [depth] * 3,
                      "box": [[64, 1, 1], [16, 8, 1], [4, 4, 4]]})
        b.run()
        b.sync()
        for (d, N, m, t), f, xx in zip(spec, fields, dev):
            e = walk.to_device(d, N, walk.step(d, m, walk.from_device(d, N, f), t))
            assert rel_l2(xx.cpu().numpy(), e) <= 1e-5, (depth, d, N)
    b.close()
