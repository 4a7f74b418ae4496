"""Serving path (qw_server_* / qw_submit / qw_poll) and the device packet builder.

* qw_prepare_packet equals the seeded generator's Gaussian packet.
* A served request's norm, <x> and particle weights equal the oracle's for the
  same normalised packet evolved to time t (complex64 tolerances).
* Each result is the same alone and inside a mix of concurrent requests.
* Admission respects the HBM budget; oversize and malformed requests are
  refused; a full queue answers QW_EAGAIN (host-side fault injection).
"""

import time

import numpy as np
import pytest

from paper_1603_06442_gb300 import inputs
from oracle import walk, spectral, observables

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def qb(qwlib):
    from paper_1603_06442_gb300 import binding
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return binding


def wait_all(qb, srv, tickets, timeout=120.0):
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t in out:
                continue
            done, obs, lat = qb.qw_poll(srv, t)
            if done:
                out[t] = (obs, lat)
        assert time.time() - t0 < timeout, "served requests did not finish"
        time.sleep(0.0005)
    return out


CHI = {1: [0.6, 0.8j], 2: [0.5, 0.5j, 0.5, -0.5j], 3: [0.6, 0.0, 0.0, 0.8j]}


@pytest.mark.parametrize("dim,N", [(1, 96), (2, 24), (3, 16), (3, 24)])
@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_device_packet_matches_generator(qb, dim, N, dtype):
    x0, sig, k0 = [N / 3 + 0.5] * dim, N / 7, [0.3, -0.2, 0.1][:dim]
    a = inputs.gaussian_packet(dim, N, x0, sig, k0, CHI[dim])
    plan = qb.Plan(dim, N, 0.1, dtype)
    x = torch.zeros(plan.elems, dtype=plan.torch_dtype, device="cuda")
    plan.prepare_packet(x, x0, sig, k0, CHI[dim])
    torch.cuda.synchronize()
    got = x.cpu().numpy().reshape(a.shape).astype(np.complex128)
    got /= np.sqrt(np.sum(np.abs(got) ** 2))
    tol = 1e-6 if dtype == "c64" else 1e-13
    assert np.linalg.norm(got - a) / np.linalg.norm(a) < tol
    plan.close()


REQS = [(1, 96, 0.1, 57), (2, 24, 0.3, 33), (3, 16, 0.2, 100), (3, 24, 0.05, 1000), (2, 18, 0.45, 7),
        (1, 1024, 0.01, 99991), (2, 48, 0.003, 100000), (3, 32, 0.3, 77777), (1, 4096, 0.0, 31),
        # x lengths with a fused x pass (weights, D_k^t and the x transforms in one kernel)
        (2, 64, 0.2, 5000), (2, 96, 0.35, 123), (3, 128, 0.15, 1000)]


def oracle_obs(dim, N, m, t, x0, sig, k0, chi):
    a = inputs.gaussian_packet(dim, N, x0, sig, k0, chi)
    psi = spectral.evolve(dim, m, walk.from_device(dim, N, a.astype(np.complex64).astype(np.complex128)), t)
    wp, wm = observables.particle_weights(dim, m, psi)
    return observables.norm(psi), observables.mean_position(dim, psi), wp, wm


def test_served_results_match_oracle(qb):
    srv = qb.qw_server_create(256 << 20, slots=4, max_pending=64)
    tickets = {}
    for dim, N, m, t in REQS:
        x0, sig, k0 = [N / 2] * dim, N / 8, [0.2] * dim
        tk = qb.qw_submit(srv, qb.make_request(dim, N, m, t, x0=x0, sigma=sig, k0=k0, chi=CHI[dim]))
        tickets[tk] = (dim, N, m, t, x0, sig, k0)
    res = wait_all(qb, srv, list(tickets))
    for tk, (dim, N, m, t, x0, sig, k0) in tickets.items():
        obs, lat = res[tk]
        nrm, xm, wp, wm = oracle_obs(dim, N, m, t, x0, sig, k0, CHI[dim])
        assert abs(obs["norm"] - nrm) < 2e-5
        for j in range(dim):
            assert abs(obs["x_mean"][j] - xm[j]) < 2e-5 * N, (dim, j)
        assert abs(obs["w_particle"] - wp) < 2e-5 and abs(obs["w_antiparticle"] - wm) < 2e-5
        assert lat > 0
    qb.qw_server_destroy(srv)


def test_same_result_alone_and_in_the_mix(qb):
    probe = (3, 128, 0.17, 4321)   # x length 64: the fused x pass
    kw = dict(x0=[64, 64, 64], sigma=8.0, k0=[0.1, 0.2, 0.0], chi=CHI[3])
    srv = qb.qw_server_create(512 << 20, slots=6, max_pending=256)
    tk = qb.qw_submit(srv, qb.make_request(*probe, **kw))
    alone = wait_all(qb, srv, [tk])[tk][0]
    rng = np.random.default_rng(3)
    tickets = []
    for i in range(40):
        if i == 17:
            probe_tk = qb.qw_submit(srv, qb.make_request(*probe, **kw))
            tickets.append(probe_tk)
            continue
        dim = int(rng.integers(1, 4))
        N = [int(rng.choice([256, 1024, 4096])), int(rng.choice([32, 48, 64])), int(rng.choice([16, 24, 48]))][dim - 1]
        tickets.append(qb.qw_submit(srv, qb.make_request(dim, N, float(rng.uniform(0, 0.5)), int(rng.integers(1, 10 ** 5)),
                                                         x0=[N / 2] * dim, sigma=N / 10, k0=[0.1] * dim,
                                                         chi=CHI[dim])))
        if i % 5 == 0:
            time.sleep(0.001)
    res = wait_all(qb, srv, tickets)
    mixed = res[probe_tk][0]
    st = qb.qw_server_stats(srv)
    assert st["completed"] >= 41 and st["peak_bytes"] <= st["budget_bytes"]
    qb.qw_server_destroy(srv)
    assert mixed["norm"] == alone["norm"]
    assert mixed["x_mean"] == alone["x_mean"]
    assert mixed["w_particle"] == alone["w_particle"]


def test_admission_by_budget(qb):
    # each BCC N=64 request needs 2*4*32^3*8 B + 2*32^3*8 B = 2.6 MB; a 6 MB pool runs at most two at once
    budget = 6 << 20
    srv = qb.qw_server_create(budget, slots=8, max_pending=1000)
    tickets = [qb.qw_submit(srv, qb.make_request(3, 64, 0.2, 10 ** 4, x0=[32] * 3, sigma=6.0, chi=CHI[3]))
               for _ in range(30)]
    peak_running = 0
    t0 = time.time()
    while qb.qw_server_stats(srv)["completed"] < 30 and time.time() - t0 < 60:
        st = qb.qw_server_stats(srv)
        peak_running = max(peak_running, st["running"])
        time.sleep(0.0002)
    res = wait_all(qb, srv, tickets)
    st = qb.qw_server_stats(srv)
    qb.qw_server_destroy(srv)
    assert st["peak_bytes"] <= budget and peak_running <= 2
    vals = {round(r[0]["x_mean"][0], 9) for r in res.values()}
    assert len(vals) == 1   # identical requests, identical answers


def test_refusals_and_queue_full(qb):
    srv = qb.qw_server_create(8 << 20, slots=1, max_pending=2)
    with pytest.raises(qb.QwError):       # not 2^a 3^b
        qb.qw_submit(srv, qb.make_request(3, 14, 0.1, 5, sigma=2.0))
    with pytest.raises(qb.QwError):       # bad dimension
        qb.qw_submit(srv, qb.make_request(4, 16, 0.1, 5, sigma=2.0))
    with pytest.raises(qb.QwError):       # larger than the whole budget
        qb.qw_submit(srv, qb.make_request(3, 128, 0.1, 5, sigma=2.0))
    saw_again = False
    tickets = []
    for _ in range(50):
        tk = qb.qw_submit(srv, qb.make_request(3, 32, 0.1, 77, x0=[16] * 3, sigma=3.0, chi=CHI[3]))
        if tk is None:
            saw_again = True
        else:
            tickets.append(tk)
    assert saw_again
    wait_all(qb, srv, tickets)
    with pytest.raises(qb.QwError):       # retired ticket
        qb.qw_poll(srv, tickets[0])
    qb.qw_server_destroy(srv)


def test_fft_tables_in_the_pool_evicted_lru(qb):
    """The FFT tables of each box size are carved from the server's pool and counted in its
    budget; when an admission needs the room, idle tables are evicted least recently used
    first, and a size whose tables were evicted gets them rebuilt with identical results.
    1D boxes: A = 2^20 (field 16 MiB + tables ~24 MiB), B = 3^12, C = 3 * 2^19 (~60 MiB with
    tables) in a 72 MiB pool: C must evict A's and B's tables, the second A must evict C's."""
    budget = 72 << 20
    srv = qb.qw_server_create(budget, slots=2, max_pending=16)
    seq = [(1 << 20, 0.2, 777), (3 ** 12, 0.1, 55), (3 << 19, 0.3, 1234), (1 << 20, 0.2, 777)]
    out = []
    for N, m, t in seq:
        tk = qb.qw_submit(srv, qb.make_request(1, N, m, t, x0=[N / 2], sigma=N / 64, k0=[0.3], chi=CHI[1]))
        out.append(wait_all(qb, srv, [tk])[tk][0])
        st = qb.qw_server_stats(srv)
        assert st["running"] == 0 and 0 < st["bytes_in_use"] <= budget   # cached tables are counted
    st = qb.qw_server_stats(srv)
    qb.qw_server_destroy(srv)
    assert st["peak_bytes"] <= budget
    assert out[3] == out[0]     # rebuilt tables, same answer
    for o in out:
        assert abs(o["norm"] - 1.0) < 1e-5
