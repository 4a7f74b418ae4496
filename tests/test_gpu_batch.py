"""GPU parity of the batched persistent launch (qw_batch_*) against the oracle and qw_step.

Every walk of a batch must end exactly where its own t updates take it
(relative L2 <= 1e-5 per 1000 steps in complex64, the stencil tolerance), for
every fusion depth and tile box; the batch runs the plain kernel's per-site
arithmetic, so its fields also equal qw_step's PLAIN results bit for bit.
"""

import numpy as np
import pytest

from paper_1603_06442_gb300 import inputs
from oracle import walk, spectral

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


def tiling(tile_sites=4096, budget=16 << 30, depth=(2, 2, 2), box2=(32, 16), box3=(8, 8, 4), box1=1024):
    return {"tile_sites": tile_sites, "l2_budget_bytes": budget, "depth": list(depth),
            "box": [[box1, 1, 1], [box2[0], box2[1], 1], list(box3)]}


TILINGS = {
    "default": None,
    "rows32_1MiB": tiling(32, 1 << 20, (1, 1, 1)),
    "rows1024_8MiB": tiling(1024, 8 << 20, (1, 1, 1)),
    "rows16384_96MiB": tiling(16384, 96 << 20, (1, 1, 1)),
    "fused2": tiling(),
    "fused3": tiling(depth=(3, 3, 3), box2=(16, 8), box3=(4, 4, 4), box1=64),
    "fused4_ragged": tiling(depth=(4, 4, 4), box2=(7, 5), box3=(3, 5, 2), box1=13),
    "box_larger_than_walk": tiling(depth=(4, 4, 2), box2=(64, 64), box3=(6, 6, 6), box1=4096),
    "mixed_depths_small_groups": tiling(512, 1 << 20, (1, 2, 3), box2=(8, 8), box3=(5, 3, 4)),
}


def test_batch_rejects_a_tile_over_shared_memory(qb):
    x = torch.zeros(4 * 64 * 64, dtype=torch.complex64, device="cuda")
    b = qb.Batch([(2, 64, 0.1, 3, x)])
    with pytest.raises(qb.QwError, match="shared memory"):
        b.set_tiling(tiling(depth=(4, 4, 4), box2=(64, 64)))     # (64 + 8)^2 x 4 x 8 B x 2 > 227 KB
    b.close()


@pytest.mark.parametrize("name", list(TILINGS))
def test_batch_matches_oracle(qb, name):
    fields = make_fields(SMALL)
    dev = [torch.from_numpy(a.astype(np.complex64)).cuda() for a in fields]
    b = qb.Batch([(d, N, m, t, x) for (d, N, m, t), x in zip(SMALL, dev)])
    if TILINGS[name] is not None:
        b.set_tiling(TILINGS[name])
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


@pytest.mark.parametrize("name", ["fused2", "fused3", "fused4_ragged", "rows1024_8MiB"])
def test_batch_bitwise_equals_plain_stencil(qb, name):
    """Fused or not, a batched walk runs the PLAIN kernel's per-site arithmetic in the same
    order: the fields agree bit for bit with qw_step's PLAIN result."""
    spec = [(1, 300, 0.2, 9), (2, 45, 0.3, 11), (2, 64, 0.1, 8), (3, 18, 0.25, 7), (3, 32, 0.4, 6)]
    fields = make_fields(spec, 7)
    dev = [torch.from_numpy(a.astype(np.complex64)).cuda() for a in fields]
    b = qb.Batch([(d, N, m, t, x) for (d, N, m, t), x in zip(spec, dev)])
    b.set_tiling(TILINGS[name])
    b.run()
    b.sync()
    for (dim, N, m, t), a, x in zip(spec, fields, dev):
        plan = qb.Plan(dim, N, m, "c64")
        plan.set_stencil("plain")
        ref = torch.from_numpy(a.astype(np.complex64)).cuda()
        plan.step(ref, t)
        plan.close()
        assert torch.equal(x, ref), (name, dim, N)
    b.close()


def test_batch_autotune_keeps_results(qb):
    fields = make_fields(SMALL, 50)
    dev = [torch.from_numpy(a.astype(np.complex64)).cuda() for a in fields]
    b = qb.Batch([(d, N, m, t, x) for (d, N, m, t), x in zip(SMALL, dev)])
    best, rate = b.autotune(rounds_cap=8)
    assert rate > 0 and all(1 <= d <= 4 for d in best["depth"])
    assert b.tiling()[0] == best
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
    worst = 0.0
    for i in rng.choice(len(mix), size=10, replace=False):
        w = mix[i]
        dim, N = w["dim"], w["N"]
        plan = qb.Plan(dim, N, w["mass"], "c64")
        plan.set_stencil("plain")
        ref = torch.from_numpy(init[i]).cuda()
        plan.step(ref, w["t"])
        plan.close()
        got = dev[i].cpu().numpy()
        assert np.array_equal(got, ref.cpu().numpy()), i   # same arithmetic as PLAIN
        # the FP64 oracle's exact Fourier evolution of the same complex64 initial field
        exp = walk.to_device(dim, N, spectral.evolve(dim, w["mass"], walk.from_device(
            dim, N, init[i].astype(np.complex128)), w["t"]))
        err = rel_l2(got.astype(np.complex128), exp)
        worst = max(worst, err / tol(w["t"]))
        print("config-4 walk %d: dim %d N %d t %d m %.3f rel-L2 vs oracle %.2e" % (i, dim, N, w["t"], w["mass"], err))
        assert err <= tol(w["t"]), (i, err)
    b.close()


def test_batch_bounded_wait_times_out_and_device_recovers(qb):
    """Fault injection: one tile never publishes its rounds, so the rounds that depend on it
    give up after a short bounded wait and qw_batch_sync reports QW_ETIMEOUT (no trap, no
    hang).  The same batch, with the stall cleared, then matches the oracle."""
    spec = [(2, 40, 0.2, 12), (3, 16, 0.3, 9), (1, 200, 0.1, 10)]
    fields = make_fields(spec, 21)
    dev = [torch.from_numpy(a.astype(np.complex64)).cuda() for a in fields]
    b = qb.Batch([(d, N, m, t, x) for (d, N, m, t), x in zip(spec, dev)])
    b.set_tiling(TILINGS["fused2"])
    b.debug_stall(0, spin_limit=4096)
    b.run()
    with pytest.raises(qb.QwError) as ei:
        b.sync()
    assert ei.value.status == qb.QW_ETIMEOUT
    b.debug_stall(-1)
    for a, x in zip(fields, dev):
        x.copy_(torch.from_numpy(a.astype(np.complex64)))
    b.run()
    b.sync()
    for (dim, N, m, t), a, x in zip(spec, fields, dev):
        exp = walk.to_device(dim, N, walk.step(dim, m, walk.from_device(dim, N, a), t))
        assert rel_l2(x.cpu().numpy(), exp) <= tol(t), (dim, N, t)
    b.close()


def test_batch_rejects_bad_walk(qb):
    x = torch.zeros(8, dtype=torch.complex64, device="cuda")
    with pytest.raises(qb.QwError):
        qb.Batch([(3, 7, 0.1, 3, x)])
    with pytest.raises(qb.QwError):
        qb.Batch([(2, 8, 1.5, 3, x)])
