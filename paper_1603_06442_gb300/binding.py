"""Thin ctypes binding of libqw.so: the C ABI of include/qw.h under the same names.

Argument marshalling only.  Fields are CUDA tensors (torch complex64 /
complex128, contiguous, device layout of include/qw.h) or raw device addresses;
streams default to torch's current stream.  Every step of the walk runs in the
CUDA library; if libqw.so is missing this module raises instead of falling back.
"""

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libqw.so")

QW_OK, QW_EINVAL, QW_ENOMEM, QW_ECUDA, QW_ETIMEOUT, QW_EAGAIN, QW_EBUSY, QW_ENOTFOUND = range(8)
QW_C64, QW_C128 = 0, 1
QW_STENCIL_AUTO, QW_STENCIL_PLAIN, QW_STENCIL_VEC, QW_STENCIL_TMA, QW_STENCIL_TMA2, QW_STENCIL_FUSED = 0, 1, 2, 3, 4, 5
STENCILS = {"auto": 0, "plain": 1, "vec": 2, "tma": 3, "tma2": 4, "fused": 5}
STATUS_NAMES = {0: "QW_OK", 1: "QW_EINVAL", 2: "QW_ENOMEM", 3: "QW_ECUDA", 4: "QW_ETIMEOUT",
                5: "QW_EAGAIN", 6: "QW_EBUSY", 7: "QW_ENOTFOUND"}


class QwError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class qw_obs(ctypes.Structure):
    _fields_ = [("norm", ctypes.c_double), ("x_mean", ctypes.c_double * 3),
                ("w_particle", ctypes.c_double), ("w_antiparticle", ctypes.c_double)]

    def as_dict(self):
        return {"norm": self.norm, "x_mean": list(self.x_mean), "w_particle": self.w_particle,
                "w_antiparticle": self.w_antiparticle}


class qw_walk(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("N", ctypes.c_int64), ("mass", ctypes.c_double), ("t", ctypes.c_int64),
                ("psi_dev", ctypes.c_void_p)]


class qw_request(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("N", ctypes.c_int64), ("mass", ctypes.c_double), ("t", ctypes.c_int64),
                ("psi0_host", ctypes.c_void_p), ("x0", ctypes.c_double * 3), ("sigma", ctypes.c_double),
                ("k0", ctypes.c_double * 3), ("chi", ctypes.c_double * 8)]


class qw_batch_tiling(ctypes.Structure):
    _fields_ = [("tile_sites", ctypes.c_int64), ("l2_budget_bytes", ctypes.c_int64), ("depth", ctypes.c_int * 3),
                ("box", (ctypes.c_int * 3) * 3)]

    def as_dict(self):
        return {"tile_sites": self.tile_sites, "l2_budget_bytes": self.l2_budget_bytes,
                "depth": list(self.depth), "box": [list(b) for b in self.box]}

    @classmethod
    def from_dict(cls, d):
        t = cls()
        t.tile_sites = int(d["tile_sites"])
        t.l2_budget_bytes = int(d["l2_budget_bytes"])
        for i in range(3):
            t.depth[i] = int(d["depth"][i])
            for a in range(3):
                t.box[i][a] = int(d["box"][i][a])
        return t


class qw_server_stats_t(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("pending", "running", "admitted", "completed", "bytes_in_use",
                                              "peak_bytes", "budget_bytes")]


_lib = None

# name -> (restype, argtypes)
_SIGS = {
    "qw_last_error": (ctypes.c_char_p, []),
    "qw_version": (ctypes.c_char_p, []),
    "qw_plan_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_void_p)]),
    "qw_plan_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "qw_plan_field_elems": (ctypes.c_int64, [ctypes.c_void_p]),
    "qw_plan_sites": (ctypes.c_int64, [ctypes.c_void_p]),
    "qw_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "qw_plan_set_stencil": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "qw_plan_get_stencil": (ctypes.c_int, [ctypes.c_void_p]),
    "qw_plan_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "qw_sync": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "qw_plan_prepare_spectral": (ctypes.c_int, [ctypes.c_void_p]),
    "qw_prepare_packet": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                         ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]),
    "qw_server_create": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "qw_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(qw_request), ctypes.POINTER(ctypes.c_uint64)]),
    "qw_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(qw_obs), ctypes.POINTER(ctypes.c_int),
                               ctypes.POINTER(ctypes.c_double)]),
    "qw_server_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(qw_server_stats_t)]),
    "qw_server_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "qw_batch_create": (ctypes.c_int, [ctypes.POINTER(qw_walk), ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "qw_batch_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "qw_batch_set_tiling": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(qw_batch_tiling)]),
    "qw_batch_get_tiling": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(qw_batch_tiling),
                                           ctypes.POINTER(ctypes.c_int64)]),
    "qw_batch_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "qw_batch_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                         ctypes.POINTER(qw_batch_tiling), ctypes.POINTER(ctypes.c_double)]),
    "qw_batch_debug_stall": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64]),
    "qw_batch_sync": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "qw_batch_observables": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(qw_obs), ctypes.c_void_p]),
    "qw_set_autotune_cache": (ctypes.c_int, [ctypes.c_char_p]),
    "qw_set_debug_poison": (ctypes.c_int, [ctypes.c_int]),
    "qw_plan_set_fusion": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "qw_plan_get_fusion": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(ctypes.c_int)]),
    "qw_plan_set_host_timing": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "qw_plan_host_timing": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int]),
    "qw_step_static": (ctypes.c_int, [ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                                      ctypes.c_int64, ctypes.c_void_p]),
    "qw_evolve_spectral": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "qw_observables": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(qw_obs),
                                      ctypes.c_void_p]),
    "qw_fw_transform": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "qw_position_moments": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                           ctypes.c_void_p]),
    "qw_projection": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p,
                                     ctypes.c_void_p]),
    "qw_projection_elems": (ctypes.c_int64, [ctypes.c_void_p, ctypes.c_int]),
    "qw_run_host": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                   ctypes.c_int, ctypes.c_int64, ctypes.POINTER(qw_obs), ctypes.c_void_p]),
}


def exported_names():
    return list(_SIGS)


def load(path=LIB_PATH):
    """Load libqw.so once; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libqw.so not found at %s: build it first (__graft_entry__.build())" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status):
    if status != QW_OK:
        raise QwError(status, load().qw_last_error().decode())


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def qw_last_error():
    return load().qw_last_error().decode()


def qw_version():
    return load().qw_version().decode()


def qw_plan_create(dim, N, mass, dtype):
    h = ctypes.c_void_p()
    _check(load().qw_plan_create(int(dim), int(N), float(mass), int(dtype), ctypes.byref(h)))
    return h.value


def qw_plan_destroy(plan):
    _check(load().qw_plan_destroy(plan))


def qw_plan_field_elems(plan):
    return load().qw_plan_field_elems(plan)


def qw_plan_sites(plan):
    return load().qw_plan_sites(plan)


def qw_step(plan, psi, nsteps, stream=None):
    _check(load().qw_step(plan, _ptr(psi), int(nsteps), _stream(stream)))


def qw_plan_set_stencil(plan, variant):
    _check(load().qw_plan_set_stencil(plan, int(STENCILS.get(variant, variant))))


def qw_plan_get_stencil(plan):
    return load().qw_plan_get_stencil(plan)


def qw_plan_prepare_spectral(plan):
    _check(load().qw_plan_prepare_spectral(plan))


def qw_evolve_spectral(plan, psi, t, stream=None):
    _check(load().qw_evolve_spectral(plan, _ptr(psi), int(t), _stream(stream)))


def _darr(vals, n):
    a = (ctypes.c_double * n)()
    for i, v in enumerate(list(vals)[:n]):
        a[i] = float(v)
    return a


def _chi8(chi):
    flat = []
    for c in chi:
        c = complex(c)
        flat += [c.real, c.imag]
    return _darr(flat + [0.0] * (8 - len(flat)), 8)


def qw_prepare_packet(plan, psi, x0, sigma, k0, chi, stream=None):
    _check(load().qw_prepare_packet(plan, _ptr(psi), _darr(list(x0) + [0, 0, 0], 3), float(sigma),
                                    _darr(list(k0) + [0, 0, 0], 3), _chi8(chi), _stream(stream)))


def qw_server_create(hbm_budget_bytes, slots=8, max_pending=4096):
    h = ctypes.c_void_p()
    _check(load().qw_server_create(int(hbm_budget_bytes), int(slots), int(max_pending), ctypes.byref(h)))
    return h.value


def make_request(dim, N, mass, t, psi0_host=None, x0=(0, 0, 0), sigma=1.0, k0=(0, 0, 0), chi=(1, 0, 0, 0)):
    r = qw_request()
    r.dim, r.N, r.mass, r.t = int(dim), int(N), float(mass), int(t)
    r.psi0_host = None if psi0_host is None else psi0_host.ctypes.data
    for i, v in enumerate((list(x0) + [0, 0, 0])[:3]):
        r.x0[i] = float(v)
    r.sigma = float(sigma)
    for i, v in enumerate((list(k0) + [0, 0, 0])[:3]):
        r.k0[i] = float(v)
    ch = _chi8(chi)
    for i in range(8):
        r.chi[i] = ch[i]
    return r


def qw_submit(server, req):
    """Returns the ticket, or None when the queue is full (QW_EAGAIN)."""
    t = ctypes.c_uint64()
    st = load().qw_submit(server, ctypes.byref(req), ctypes.byref(t))
    if st == QW_EAGAIN:
        return None
    _check(st)
    return t.value


def qw_poll(server, ticket):
    """(done, obs dict or None, latency seconds or None)."""
    o, d, lat = qw_obs(), ctypes.c_int(), ctypes.c_double()
    _check(load().qw_poll(server, int(ticket), ctypes.byref(o), ctypes.byref(d), ctypes.byref(lat)))
    return (True, o.as_dict(), lat.value) if d.value else (False, None, None)


def qw_server_stats(server):
    s = qw_server_stats_t()
    _check(load().qw_server_stats(server, ctypes.byref(s)))
    return {n: getattr(s, n) for n, _ in qw_server_stats_t._fields_}


def qw_server_destroy(server):
    _check(load().qw_server_destroy(server))


def qw_set_debug_poison(on):
    _check(load().qw_set_debug_poison(1 if on else 0))


def qw_set_autotune_cache(path):
    _check(load().qw_set_autotune_cache(path.encode() if path else None))


def qw_plan_set_fusion(plan, depth, box):
    b = (ctypes.c_int * 3)(*[int(v) for v in (list(box) + [1, 1, 1])[:3]])
    _check(load().qw_plan_set_fusion(plan, int(depth), b))


def qw_plan_get_fusion(plan):
    d, b = ctypes.c_int(), (ctypes.c_int * 3)()
    _check(load().qw_plan_get_fusion(plan, ctypes.byref(d), b))
    return d.value, list(b)


def qw_plan_set_host_timing(plan, on):
    _check(load().qw_plan_set_host_timing(plan, 1 if on else 0))


def qw_plan_host_timing(plan, count):
    """[(copy_start, copy_end, step_start, step_end, obs_end) in ms] for the last timed run."""
    out = (ctypes.c_double * (5 * count))()
    _check(load().qw_plan_host_timing(plan, out, int(count)))
    return [tuple(out[5 * j:5 * j + 5]) for j in range(count)]


def qw_step_static(dim, N, mass, dtype, psi, nsteps, stream=None):
    dt = QW_C64 if dtype in ("c64", QW_C64) else QW_C128
    _check(load().qw_step_static(int(dim), int(N), float(mass), dt, _ptr(psi), int(nsteps), _stream(stream)))


def qw_plan_autotune(plan, stream=None):
    r = ctypes.c_double()
    _check(load().qw_plan_autotune(plan, _stream(stream), ctypes.byref(r)))
    return r.value


def qw_sync(plan, stream=None):
    _check(load().qw_sync(plan, _stream(stream)))


def qw_observables(plan, psi, stream=None):
    out = qw_obs()
    _check(load().qw_observables(plan, _ptr(psi), ctypes.byref(out), _stream(stream)))
    return out.as_dict()


def qw_fw_transform(plan, psi, out, stream=None):
    _check(load().qw_fw_transform(plan, _ptr(psi), _ptr(out), _stream(stream)))


def qw_position_moments(plan, psi, stream=None):
    """{'norm', 'mean' (3), 'cov' (3x3 nested lists)} of the density."""
    out = (ctypes.c_double * 10)()
    _check(load().qw_position_moments(plan, _ptr(psi), out, _stream(stream)))
    c = list(out)
    xx, yy, zz, xy, xz, yz = c[4:10]
    return {"norm": c[0], "mean": c[1:4], "cov": [[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]]}


def keep_mask(keep):
    """Axis set (0 = x, 1 = y, 2 = z) or int mask -> int mask."""
    if isinstance(keep, int):
        return keep
    m = 0
    for a in keep:
        m |= 1 << int(a)
    return m


def qw_projection_elems(plan, keep):
    return int(load().qw_projection_elems(plan, keep_mask(keep)))


def qw_projection(plan, psi, keep, out, stream=None):
    _check(load().qw_projection(plan, _ptr(psi), keep_mask(keep), _ptr(out), _stream(stream)))


def _host_ptr(x):
    """Address of a host buffer: a CPU torch tensor, a numpy array or an int."""
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if x.is_cuda:
            raise ValueError("qw_run_host takes host buffers")
        return x.data_ptr()
    return x.ctypes.data


def qw_run_host(plan, fields, nsteps, out_fields=None, stream=None):
    """Copy each host field to the device, advance it nsteps and return its observables
    (one dict per field); out_fields (optional) receive the evolved fields."""
    n = len(fields)
    ins = (ctypes.c_void_p * max(n, 1))(*[_host_ptr(f) for f in fields])
    outs = None
    if out_fields is not None:
        if len(out_fields) != n:
            raise ValueError("out_fields must match fields")
        outs = (ctypes.c_void_p * max(n, 1))(*[_host_ptr(f) for f in out_fields])
    res = (qw_obs * max(n, 1))()
    _check(load().qw_run_host(plan, ins, outs, n, int(nsteps), res, _stream(stream)))
    return [res[j].as_dict() for j in range(n)]


def qw_batch_create(walks):
    """walks: list of (dim, N, mass, t, field tensor or device address)."""
    arr = (qw_walk * len(walks))()
    for i, (dim, N, mass, t, psi) in enumerate(walks):
        arr[i] = qw_walk(int(dim), int(N), float(mass), int(t), _ptr(psi))
    h = ctypes.c_void_p()
    _check(load().qw_batch_create(arr, len(walks), ctypes.byref(h)))
    return h.value


def qw_batch_destroy(batch):
    _check(load().qw_batch_destroy(batch))


def qw_batch_set_tiling(batch, tiling):
    """tiling: dict with tile_sites, l2_budget_bytes, depth (3 ints) and box (3 x 3 ints)."""
    t = qw_batch_tiling.from_dict(tiling)
    _check(load().qw_batch_set_tiling(batch, ctypes.byref(t)))


def qw_batch_get_tiling(batch):
    """(tiling dict, work items of one run)."""
    t, items = qw_batch_tiling(), ctypes.c_int64()
    _check(load().qw_batch_get_tiling(batch, ctypes.byref(t), ctypes.byref(items)))
    return t.as_dict(), items.value


def qw_batch_run(batch, stream=None):
    _check(load().qw_batch_run(batch, _stream(stream)))


def qw_batch_autotune(batch, rounds_cap=32, stream=None):
    """(chosen tiling dict, its measured site-steps/s)."""
    t, r = qw_batch_tiling(), ctypes.c_double()
    _check(load().qw_batch_autotune(batch, int(rounds_cap), _stream(stream), ctypes.byref(t), ctypes.byref(r)))
    return t.as_dict(), r.value


def qw_batch_debug_stall(batch, walk, spin_limit=0):
    _check(load().qw_batch_debug_stall(batch, int(walk), int(spin_limit)))


def qw_batch_sync(batch, stream=None):
    _check(load().qw_batch_sync(batch, _stream(stream)))


def qw_batch_observables(batch, n, stream=None):
    out = (qw_obs * n)()
    _check(load().qw_batch_observables(batch, out, _stream(stream)))
    return [o.as_dict() for o in out]


class Batch:
    """Owning wrapper of a qw_batch over (dim, N, mass, t, field) walks (complex64)."""

    def __init__(self, walks):
        self.walks = list(walks)
        self.handle = qw_batch_create(self.walks)

    def run(self, stream=None):
        qw_batch_run(self.handle, stream)

    def sync(self, stream=None):
        qw_batch_sync(self.handle, stream)

    def autotune(self, rounds_cap=32, stream=None):
        return qw_batch_autotune(self.handle, rounds_cap, stream)

    def set_tiling(self, tiling):
        qw_batch_set_tiling(self.handle, tiling)

    def tiling(self):
        return qw_batch_get_tiling(self.handle)

    def debug_stall(self, walk, spin_limit=0):
        qw_batch_debug_stall(self.handle, walk, spin_limit)

    def observables(self, stream=None):
        return qw_batch_observables(self.handle, len(self.walks), stream)

    def close(self):
        if getattr(self, "handle", None):
            qw_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """Owning wrapper of a qw_plan (destroyed with the object)."""

    def __init__(self, dim, N, mass, dtype="c64"):
        self.dim, self.N, self.mass = int(dim), int(N), float(mass)
        self.dtype = QW_C64 if dtype in ("c64", QW_C64) else QW_C128
        self.handle = qw_plan_create(self.dim, self.N, self.mass, self.dtype)
        self.elems = qw_plan_field_elems(self.handle)
        self.sites = qw_plan_sites(self.handle)

    @property
    def torch_dtype(self):
        import torch
        return torch.complex64 if self.dtype == QW_C64 else torch.complex128

    def field_shape(self):
        N = self.N
        if self.dim == 1:
            return (2, N)
        if self.dim == 2:
            return (4, N, N)
        M = N // 2
        return (2, 4, M, M, M)

    def check_field(self, psi):
        if not psi.is_cuda or not psi.is_contiguous() or psi.dtype != self.torch_dtype \
                or psi.numel() != self.elems:
            raise ValueError("field must be a contiguous CUDA %s tensor with %d elements"
                             % (self.torch_dtype, self.elems))

    def step(self, psi, nsteps, stream=None):
        self.check_field(psi)
        qw_step(self.handle, psi, nsteps, stream)

    def autotune(self, stream=None):
        return qw_plan_autotune(self.handle, stream)

    def set_stencil(self, variant):
        qw_plan_set_stencil(self.handle, variant)

    @property
    def stencil(self):
        return qw_plan_get_stencil(self.handle)

    def prepare_spectral(self):
        qw_plan_prepare_spectral(self.handle)

    def evolve_spectral(self, psi, t, stream=None):
        self.check_field(psi)
        qw_evolve_spectral(self.handle, psi, t, stream)

    def sync(self, stream=None):
        qw_sync(self.handle, stream)

    def prepare_packet(self, psi, x0, sigma, k0, chi, stream=None):
        self.check_field(psi)
        qw_prepare_packet(self.handle, psi, x0, sigma, k0, chi, stream)

    def observables(self, psi, stream=None):
        self.check_field(psi)
        return qw_observables(self.handle, psi, stream)

    def fw_transform(self, psi, out=None, stream=None):
        """Foldy-Wouthuysen field of psi (a new CUDA tensor unless `out` is given)."""
        import torch
        self.check_field(psi)
        if out is None:
            out = torch.empty_like(psi)
        self.check_field(out)
        qw_fw_transform(self.handle, psi, out, stream)
        return out

    def position_moments(self, psi, stream=None):
        self.check_field(psi)
        return qw_position_moments(self.handle, psi, stream)

    def projection(self, psi, keep, stream=None):
        """Density summed over the axes not in `keep` (axis set or mask): a CUDA float64
        tensor shaped (N,) * kept axes, indexed [z][y][x] over the kept ones."""
        import torch
        self.check_field(psi)
        mask = keep_mask(keep)
        n = qw_projection_elems(self.handle, mask)
        if n < 0:
            raise ValueError("bad keep mask %r for dim %d" % (keep, self.dim))
        kept = bin(mask).count("1")
        out = torch.empty((self.N,) * kept, dtype=torch.float64, device=psi.device)
        qw_projection(self.handle, psi, mask, out, stream)
        return out

    def check_host_field(self, f):
        if hasattr(f, "is_cuda"):
            ok = (not f.is_cuda) and f.is_contiguous() and f.dtype == self.torch_dtype and f.numel() == self.elems
        else:
            import numpy as np
            want = np.complex64 if self.dtype == QW_C64 else np.complex128
            ok = f.dtype == want and f.flags["C_CONTIGUOUS"] and f.size == self.elems
        if not ok:
            raise ValueError("host field must be a contiguous CPU %s array with %d elements"
                             % (self.torch_dtype, self.elems))

    def run_host(self, fields, nsteps, out_fields=None, stream=None):
        """End to end on host fields (page-locked copies overlap): see qw_run_host."""
        for f in list(fields) + list(out_fields or []):
            self.check_host_field(f)
        return qw_run_host(self.handle, fields, nsteps, out_fields, stream)

    def set_fusion(self, depth, box):
        qw_plan_set_fusion(self.handle, depth, box)

    def fusion(self):
        return qw_plan_get_fusion(self.handle)

    def set_host_timing(self, on=True):
        qw_plan_set_host_timing(self.handle, on)

    def host_timing(self, count):
        return qw_plan_host_timing(self.handle, count)

    def close(self):
        if getattr(self, "handle", None):
            qw_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
