"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

Holds none of the walk's arithmetic: only lattice geometry (where the sites of
the device layout sit), seeded random numbers, and plain Gaussian envelopes.
Every field is returned as a complex128 numpy array in the device layout of
include/qw.h (components planar, x fastest; BCC as two cosets), normalised to
sum |psi|^2 = 1.

Recipes (shaped like the paper's runs, Sec. 5, Figs. 2-6):
* ``gaussian_packet``: psi(x) = exp(-|d|^2 / (4 sigma^2)) exp(i k0.d) chi, with d
  the minimum-image displacement from x0 on the periodic box and chi a fixed
  spinor (|psi|^2 has standard deviation sigma sites per axis).
* ``random_field``: i.i.d. complex normal amplitudes on every lattice site.
* ``localized``: one site, one spinor (Figs. 3, 4).
* workload samplers for the batched and served mixes.
"""

import numpy as np

__all__ = ["field_shape", "n_components", "site_positions", "gaussian_packet", "random_packets", "random_field",
           "localized", "sample_batch_mix", "sample_served_stream", "snap_fft_size"]


def n_components(dim):
    return 2 if dim == 1 else 4


def field_shape(dim, N):
    if dim == 1:
        return (2, N)
    if dim == 2:
        return (4, N, N)
    if N % 2:
        raise ValueError("BCC box side N must be even")
    M = N // 2
    return (2, 4, M, M, M)


def site_positions(dim, N):
    """Coordinates of every site of the device layout, one array per axis.

    dim 1: shape (N,); dim 2: (N, N) as [y][x]; dim 3: (2, M, M, M) as
    [coset][z][y][x] with position 2*(x, y, z) + coset*(1, 1, 1).
    """
    if dim == 1:
        return [np.arange(N, dtype=float)]
    if dim == 2:
        y, x = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
        return [x.astype(float), y.astype(float)]
    M = N // 2
    c, z, y, x = np.meshgrid(np.arange(2), np.arange(M), np.arange(M), np.arange(M), indexing="ij")
    return [2.0 * x + c, 2.0 * y + c, 2.0 * z + c]


def _normalise(a):
    return a / np.sqrt(np.sum(np.abs(a) ** 2))


def gaussian_packet(dim, N, x0, sigma, k0, spinor):
    """Gaussian envelope times plane wave times a fixed spinor, device layout."""
    pos = site_positions(dim, N)
    x0 = np.broadcast_to(np.asarray(x0, dtype=float), (dim,))
    k0 = np.broadcast_to(np.asarray(k0, dtype=float), (dim,))
    r2 = 0.0
    phase = 0.0
    for j in range(dim):
        d = (pos[j] - x0[j] + N / 2.0) % N - N / 2.0
        r2 = r2 + d * d
        phase = phase + k0[j] * d
    env = np.exp(-r2 / (4.0 * sigma * sigma)) * np.exp(1j * phase)
    chi = np.asarray(spinor, dtype=complex)
    s = n_components(dim)
    if chi.shape != (s,):
        raise ValueError("spinor must have %d components" % s)
    if dim == 3:
        out = env[:, None] * chi[None, :, None, None, None]
    else:
        out = chi.reshape((s,) + (1,) * dim) * env[None]
    return _normalise(out.astype(complex))


def random_packets(dim, N, n_packets, sigma, kmax, seed, spinor=None):
    """Superposition of Gaussian packets: centres uniform in the box, wave-vector
    directions uniform, |k0| ~ U[0, kmax], phases U[0, 2 pi), fixed spinor."""
    rng = np.random.default_rng(seed)
    s = n_components(dim)
    chi = np.asarray(spinor if spinor is not None else ([1, 0] if dim == 1 else [0.5, 0.5, 0.5, 0.5]), complex)
    out = np.zeros(field_shape(dim, N), dtype=complex)
    for _ in range(n_packets):
        x0 = rng.uniform(0, N, size=dim)
        if dim == 3:
            x0 = 2.0 * np.round(x0 / 2.0)          # a BCC site of coset 0
        d = rng.normal(size=dim)
        d /= np.linalg.norm(d)
        k0 = d * rng.uniform(0.0, kmax)
        ph = np.exp(1j * rng.uniform(0, 2 * np.pi))
        out = out + ph * gaussian_packet(dim, N, x0, sigma, k0, chi)
    return _normalise(out)


def random_field(dim, N, seed):
    rng = np.random.default_rng(seed)
    shp = field_shape(dim, N)
    a = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    return _normalise(a)


def localized(dim, N, site, spinor):
    """One lattice site (device-layout index without the component axis)."""
    out = np.zeros(field_shape(dim, N), dtype=complex)
    chi = np.asarray(spinor, dtype=complex)
    if dim == 3:
        c, z, y, x = site
        out[c, :, z, y, x] = chi
    elif dim == 2:
        y, x = site
        out[:, y, x] = chi
    else:
        out[:, site[0]] = chi
    return _normalise(out)


def snap_fft_size(v):
    """Nearest integer of the form 2^a 3^b (>= 2) to v, in log distance."""
    best, bd = 2, float("inf")
    a = 1
    while a <= 1 << 20:
        b = a
        while b <= 1 << 21:
            if b >= 2:
                d = abs(np.log(b) - np.log(v))
                if d < bd:
                    best, bd = b, d
            b *= 3
        a *= 2
    return best


def sample_batch_mix(n_walks=256, seed=0):
    """Uneven walk mix: 2D square N ~ log-U[64, 1024], BCC N ~ 2*round(log-U[32, 128]/2),
    m ~ U[0, 0.5], t ~ U{100..5000}; packets of width N/16 at the box centre."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_walks):
        if rng.random() < 0.5:
            dim, N = 2, int(round(np.exp(rng.uniform(np.log(64), np.log(1024)))))
        else:
            dim, N = 3, 2 * int(round(np.exp(rng.uniform(np.log(32), np.log(128))) / 2))
        out.append({"dim": dim, "N": N, "mass": float(rng.uniform(0.0, 0.5)),
                    "t": int(rng.integers(100, 5001)), "sigma": N / 16.0})
    return out


def sample_served_stream(n_req=2000, rate=200.0, seed=0):
    """Poisson arrivals; dim ~ U{1,2,3}; sites ~ log-U[1e4, 1e8] snapped to FFT sizes;
    m ~ U[0, 0.5]; t = round(log-U[10, 1e5])."""
    rng = np.random.default_rng(seed)
    t_arr = np.cumsum(rng.exponential(1.0 / rate, size=n_req))
    out = []
    for i in range(n_req):
        dim = int(rng.integers(1, 4))
        S = float(np.exp(rng.uniform(np.log(1e4), np.log(1e8))))
        if dim == 1:
            N = snap_fft_size(S)
        elif dim == 2:
            N = snap_fft_size(np.sqrt(S))
        else:
            N = 2 * snap_fft_size((S / 2.0) ** (1.0 / 3.0))
        out.append({"arrival": float(t_arr[i]), "dim": dim, "N": int(N),
                    "mass": float(rng.uniform(0.0, 0.5)),
                    "t": int(round(np.exp(rng.uniform(np.log(10), np.log(1e5)))))})
    return out
