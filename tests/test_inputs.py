"""Host-side input generators: shapes, normalisation, placement, seeding."""

import numpy as np

from paper_1603_06442_gb300 import inputs
from oracle import walk


def test_shapes_and_norm():
    for dim, N in ((1, 10), (2, 6), (3, 8)):
        a = inputs.random_field(dim, N, 0)
        assert a.shape == inputs.field_shape(dim, N)
        assert abs(np.sum(np.abs(a) ** 2) - 1) < 1e-12
        assert np.array_equal(a, inputs.random_field(dim, N, 0))


def test_packet_centre_and_width():
    N, sig = 64, 5.0
    a = inputs.gaussian_packet(3, N, (20, 30, 40), sig, (0.1, 0, 0), [1, 0, 0, 0])
    psi = walk.from_device(3, N, a)
    dens = np.sum(np.abs(psi) ** 2, axis=0)
    coords = walk.site_coordinates(3, N)
    disp = [(c - x0 + N / 2) % N - N / 2 for c, x0 in zip(coords, (20, 30, 40))]
    assert np.allclose([np.sum(d * dens) for d in disp], 0.0, atol=1e-6)
    var = np.sum((coords[0] - 20) ** 2 * dens)
    assert abs(np.sqrt(var) - sig) < 0.05 * sig


def test_bcc_positions_match_oracle_layout():
    N = 6
    pos = inputs.site_positions(3, N)
    a = np.zeros(inputs.field_shape(3, N), dtype=complex)
    a[1, 2, 0, 2, 1] = 1.0          # coset 1, comp 2, z=0, y=2, x=1
    psi = walk.from_device(3, N, a)
    x, y, z = (int(p[1, 0, 2, 1]) for p in pos)
    assert psi[2, x, y, z] == 1.0


def test_snap_and_mixes():
    assert inputs.snap_fft_size(100) in (96, 108)
    assert inputs.snap_fft_size(1000) == 1024
    mix = inputs.sample_batch_mix(256, 0)
    assert len(mix) == 256 and all(w["dim"] in (2, 3) for w in mix)
    assert all(w["N"] % 2 == 0 for w in mix if w["dim"] == 3)
    st = inputs.sample_served_stream(100, 200.0, 0)
    assert all(b["arrival"] > a["arrival"] for a, b in zip(st, st[1:]))
