"""GPU parity of qw_run_host: host fields copied in, advanced by the update rule (Eq. upd-rule),
observables and evolved fields back on the host, checked against the oracle field by field.

Tolerances as for qw_step / qw_observables: relative L2 1e-11 (complex128) and 1e-5 (complex64)
on the fields; norm and mean position to 1e-12 / 1e-6 relative; particle weights 1e-12 / 2e-6.
"""

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


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = [(d, N, dt, t) for (d, N) in [(1, 64), (2, 24), (2, 64), (3, 16), (3, 42)]
         for dt in ("c128", "c64") for t in (0, 5, 6)]
# BCC N=128 (x length 64): the complex64 observables take the fused x-pass weights kernel
CASES += [(3, 128, "c64", 6)]


@pytest.mark.parametrize("dim,N,dtype,t", CASES)
def test_run_host_matches_oracle(qb, dim, N, dtype, t):
    npdt = np.complex64 if dtype == "c64" else np.complex128
    m = 0.3
    count = 7  # every one of the three device buffers and both observables stages reused
    fields = [np.ascontiguousarray(inputs.random_field(dim, N, seed=70 + j).astype(npdt)) for j in range(count)]
    # one pageable numpy field, the others page-locked torch tensors
    hosts = [fields[0]] + [torch.from_numpy(f.copy()).pin_memory() for f in fields[1:]]
    outs = [np.zeros_like(f) for f in fields]
    plan = qb.Plan(dim, N, m, dtype)
    res = plan.run_host(hosts, t, out_fields=outs)
    plan.close()
    assert len(res) == count
    ftol = 1e-11 if dtype == "c128" else 1e-5
    rtol = 1e-12 if dtype == "c128" else 1e-6
    wtol = 1e-12 if dtype == "c128" else 2e-6
    kspace = all(inputs.snap_fft_size(L) == L for L in ([N] if dim < 3 else [N // 2]))
    for j in range(count):
        psi0 = walk.from_device(dim, N, fields[j])
        psi_t = walk.step(dim, m, psi0, t)
        exp = walk.to_device(dim, N, psi_t)
        err = rel_l2(outs[j].astype(np.complex128), exp)
        assert err <= ftol, (j, err)
        nrm = observables.norm(psi_t)
        assert abs(res[j]["norm"] - nrm) <= rtol * nrm
        xm = observables.mean_position(dim, psi_t)
        for k in range(dim):
            assert abs(res[j]["x_mean"][k] - xm[k]) <= rtol * N, (j, k)
        if kspace:
            wp, wm = observables.particle_weights(dim, m, psi_t)
            assert abs(res[j]["w_particle"] - wp) <= wtol
            assert abs(res[j]["w_antiparticle"] - wm) <= wtol
    # the input fields are left as they were
    np.testing.assert_array_equal(fields[0], inputs.random_field(dim, N, seed=70).astype(npdt))


def test_run_host_in_place_and_single_field(qb):
    """psi_out_host may be the input buffer itself; a single field takes the same path."""
    dim, N, m, t = 3, 64, 0.1, 4
    a = np.ascontiguousarray(inputs.random_field(dim, N, seed=3).astype(np.complex64))
    exp = walk.to_device(dim, N, walk.step(dim, m, walk.from_device(dim, N, a), t))
    buf = torch.from_numpy(a.copy()).pin_memory()
    plan = qb.Plan(dim, N, m, "c64")
    res = plan.run_host([buf], t, out_fields=[buf])
    # a second call reuses the plan's device buffers
    res2 = plan.run_host([a], t)
    plan.close()
    assert rel_l2(buf.numpy().astype(np.complex128), exp) <= 1e-5
    assert abs(res[0]["norm"] - res2[0]["norm"]) <= 1e-6 * res2[0]["norm"]


def test_run_host_rejects_bad_arguments(qb):
    plan = qb.Plan(2, 8, 0.1, "c64")
    f = np.zeros(plan.elems, dtype=np.complex64)
    assert qb.qw_run_host(plan.handle, [], 3) == []
    with pytest.raises(qb.QwError):
        qb.qw_run_host(plan.handle, [f], -1)
    with pytest.raises(qb.QwError):
        qb.qw_run_host(plan.handle, [0], 1)
    with pytest.raises(ValueError):
        plan.run_host([np.zeros(plan.elems, dtype=np.complex128)], 1)
    with pytest.raises(ValueError):
        plan.run_host([torch.zeros(plan.elems, dtype=torch.complex64, device="cuda")], 1)
    plan.close()


def test_host_run_timing_timeline(qb):
    """qw_plan_set_host_timing / qw_plan_host_timing: per field, the copy precedes the step
    (the step waits for its field), the observables follow the step, and the copy of field
    j + 1 starts no later than field j's step ends (it overlaps)."""
    dim, N, m = 3, 64, 0.2
    plan = qb.Plan(dim, N, m, "c64")
    a = inputs.random_field(dim, N, seed=4).astype(np.complex64)
    host = [torch.from_numpy(a).pin_memory() for _ in range(4)]
    plan.set_host_timing(True)
    plan.run_host(host, 6)
    tl = plan.host_timing(4)
    plan.set_host_timing(False)
    with pytest.raises(qb.QwError):
        plan.host_timing(5)
    plan.close()
    for j, (c0, c1, s0, s1, o1) in enumerate(tl):
        assert 0.0 <= c0 <= c1 <= s0 <= s1 <= o1, (j, tl[j])
        if j + 1 < len(tl):
            assert tl[j + 1][0] <= s1, (j, tl)
