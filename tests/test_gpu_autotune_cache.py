"""qw_set_autotune_cache: the plan and batch autotuners reuse a recorded choice for the same
GPU model and problem instead of measuring again, and record what they measure."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def qb(qwlib):
    from paper_1603_06442_gb300 import binding
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return binding


def test_plan_autotune_cache(qb, tmp_path):
    path = tmp_path / "tune.txt"
    qb.qw_set_autotune_cache(str(path))
    try:
        plan = qb.Plan(2, 64, 0.2, "c64")
        r1 = plan.autotune()
        v1, f1 = plan.stencil, plan.fusion()
        plan.close()
        lines = path.read_text().splitlines()
        assert len(lines) == 1 and lines[0].startswith("plan ") and "dim=2 N=64 dtype=c64 |" in lines[0]
        plan = qb.Plan(2, 64, 0.2, "c64")
        r2 = plan.autotune()
        assert (plan.stencil, plan.fusion(), r2) == (v1, f1, r1)
        plan.close()
        assert len(path.read_text().splitlines()) == 1      # a hit appends nothing
        # the last matching line wins: a recorded PLAIN choice is applied as it stands
        path.write_text(lines[0] + "\n" + lines[0].split("|")[0] + "| 1 0 0 0 0 123\n")
        plan = qb.Plan(2, 64, 0.2, "c64")
        assert plan.autotune() == 123.0 and plan.stencil == qb.STENCILS["plain"]
        plan.close()
        plan = qb.Plan(2, 48, 0.2, "c64")                    # another problem: measured, appended
        plan.autotune()
        plan.close()
        assert len(path.read_text().splitlines()) == 3
    finally:
        qb.qw_set_autotune_cache(None)


def test_batch_autotune_cache(qb, tmp_path):
    path = tmp_path / "tune.txt"
    qb.qw_set_autotune_cache(str(path))
    try:
        spec = [(2, 40, 0.2, 30), (3, 16, 0.3, 20), (1, 200, 0.1, 25)]
        fields = [torch.zeros(4 * 40 * 40, dtype=torch.complex64, device="cuda"),
                  torch.zeros(2 * 4 * 8 ** 3, dtype=torch.complex64, device="cuda"),
                  torch.zeros(2 * 200, dtype=torch.complex64, device="cuda")]
        b = qb.Batch([(d, N, m, t, x) for (d, N, m, t), x in zip(spec, fields)])
        t1, r1 = b.autotune(rounds_cap=8)
        b.close()
        assert len(path.read_text().splitlines()) == 1
        b = qb.Batch([(d, N, m, t, x) for (d, N, m, t), x in zip(spec, fields)])
        t2, r2 = b.autotune(rounds_cap=8)
        assert (t2, r2) == (t1, r1) and b.tiling()[0] == t1
        b.close()
        assert len(path.read_text().splitlines()) == 1
    finally:
        qb.qw_set_autotune_cache(None)
