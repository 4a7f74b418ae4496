"""GPU parity of the batched persistent launch (qw_batch_*) against the oracle and qw_step.

Every walk of a batch must end exactly where its own t updates take it
(relative L2 <= 1e-5 per 1000 steps in complex64, the stencil tolerance).
"""

import numpy as np
import pytest

from paper_1603_06442_gb300 import inputs
from oracle import walk

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def tol(t):
    return 1e-5 * max(1.0, t / 1000.0)


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def qb(qwlib):
    from paper_1603_06442_gb300 import binding
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return binding


SMALL = [(1, 64, 0.1, 5), (1, 1000, 0.3, 0), (1, 37, 0.2, 8), (2, 24, 0.2, 7), (2, 40, 0.45, 12),
         (2, 9, 0.0, 3), (3, 8, 0.05, 3), (3, 20, 0.3, 10), (3, 12, 1.0, 4), (3, 34, 0.25, 1)]


def make_fields(spec, seed0=0):
    out = []
    for i, (dim, N, m, t) in enumerate(spec):
        a = inputs.random_field(dim, N, seed=seed0 + i)
        out.append(a)
    return out


@pytest.mark.parametrize("tiling", [None, (32, 1 << 20), (1024, 8 << 20), (16384, 96 << 20)])
def test_batch_matches_oracle(qb, tiling):
    fields = make_fields(SMALL)
    dev = [torch.from_numpy(a.astype(np.complex64)).cuda() for a in fields]
    b = qb.Batch([(d, N, m, t, x) for (d, N, m, t), x in zip(SMALL, dev)])
    if tiling is not None:
        b.set_tiling(*tiling)
    b.run()
    b.sync()
    for (dim, N, m, t), a, x in zip(SMALL, fields, dev):
        exp = walk.to_device(dim, N, walk.step(dim, m, walk.from_device(dim, N, a), t))
        assert rel_l2(x.cpu().numpy(), exp) <= tol(t), (dim, N, t)
    # graph replay: a second run advances every walk by t again
    b.run()
    b.sync()
    for (dim, N, m, t), a, x in zip(SMALL, fields, dev):
        exp = walk.to_device(dim, N, walk.step(dim, m, walk.from_device(dim, N, a), 2 * t))
        assert rel_l2(x.cpu().numpy(), exp) <= tol(2 * t), (dim, N, t)
    obs = b.observables()
    for (dim, N, m, t), x, o in zip(SMALL, dev, obs):
        plan = qb.Plan(dim, N, m, "c64")
        ref = plan.observables(x)
        plan.close()
        assert abs(o["norm"] - ref["norm"]) < 1e-6
        assert all(abs(o["x_mean"][j] - ref["x_mean"][j]) < 1e-6 * N for j in range(3))
    b.close()


def test_batch_autotune_keeps_results(qb):
    fields = make_fields(SMALL, 50)
    dev = [torch.from_numpy(a.astype(np.complex64)).cuda() for a in fields]
    b = qb.Batch([(d, N, m, t, x) for (d, N, m, t), x in zip(SMALL, dev)])
    tile, budget, rate = b.autotune(rounds_cap=8)
    assert tile in (1024, 2048, 4096, 8192, 16384) and rate > 0
    # the autotuner works on stand-in fields: the walks' own fields are untouched
    for a, x in zip(fields, dev):
        assert np.array_equal(x.cpu().numpy(), a.astype(np.complex64))
    b.run()
    b.sync()
    for (dim, N, m, t), a, x in zip(SMALL, fields, dev):
        exp = walk.to_device(dim, N, walk.step(dim, m, walk.from_device(dim, N, a), t))
        assert rel_l2(x.cpu().numpy(), exp) <= tol(t)
    b.close()


def test_batch_config_mix_256(qb):
    """256 walks: 2D N log-U[64, 1024] and BCC N log-U[32, 128], m U[0, 0.5], t U{100..5000}."""
    mix = inputs.sample_batch_mix(256, seed=0)
    rng = np.random.default_rng(1)
    dev, init = [], []
    for w in mix:
        N = w["N"]
        a = inputs.gaussian_packet(w["dim"], N, [N / 2] * w["dim"], w["sigma"], [0.0] * w["dim"],
                                   [0.5, 0.5, 0.5j, -0.5j]).astype(np.complex64)
        init.append(a)
        dev.append(torch.from_numpy(a).cuda())
    b = qb.Batch([(w["dim"], w["N"], w["mass"], w["t"], x) for w, x in zip(mix, dev)])
    b.run()
    b.sync()
    for i in rng.choice(len(mix), size=10, replace=False):
        w = mix[i]
        plan = qb.Plan(w["dim"], w["N"], w["mass"], "c64")
        plan.set_stencil("plain")
        ref = torch.from_numpy(init[i]).cuda()
        plan.step(ref, w["t"])
        plan.close()
        assert rel_l2(dev[i].cpu().numpy(), ref.cpu().numpy()) <= 1e-6, i
    b.close()


def test_batch_rejects_bad_walk(qb):
    x = torch.zeros(8, dtype=torch.complex64, device="cuda")
    with pytest.raises(qb.QwError):
        qb.Batch([(3, 7, 0.1, 3, x)])
    with pytest.raises(qb.QwError):
        qb.Batch([(2, 8, 1.5, 3, x)])
