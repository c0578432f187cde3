"""Python binding of the srdr C ABI (include/srdr.h): argument marshalling only.

Every step of the relaxation runs in the CUDA library ``_build/libsrdr.so``;
this module only converts numpy arrays and descriptions to the C types.  It
raises if the library cannot be loaded: there is no CPU fallback.

The functions keep the C names.  ``Body`` is a small owning wrapper around a
``srdr_body*`` handle.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libsrdr.so")

SRDR_PASS_AUTO = 0
SRDR_PASS_SELL = 1
SRDR_PASS_BRICKS = 2
SRDR_PASS_STENCIL = 3
SRDR_PASS_LAYOUT_AUTO, SRDR_PASS_LAYOUT_SELL = 0, 1
SRDR_SWEEP_AUTO = 0
SRDR_SWEEP_BARRIER = 1
SRDR_SWEEP_CELLS = 2
SRDR_OK = 0
SRDR_ERR_INVALID = -1
SRDR_ERR_NO_MEMORY = -2
SRDR_ERR_CUDA = -3
SRDR_ERR_NOT_CONVERGED = -4
SRDR_ERR_NONFINITE = -5
SRDR_ERR_TIMEOUT = -6
SRDR_ERR_BUSY = -7
STATUS_NAMES = {0: "OK", -1: "INVALID", -2: "NO_MEMORY", -3: "CUDA", -4: "NOT_CONVERGED",
                -5: "NONFINITE", -6: "TIMEOUT", -7: "BUSY"}

SRDR_LINEAR_SVK, SRDR_NEO_HOOKEAN = 0, 1
SRDR_FP64, SRDR_FP32_MIXED = 0, 1
SRDR_DAMP_NONE, SRDR_DAMP_PARTICLE, SRDR_DAMP_PAIRWISE, SRDR_DAMP_EXPLICIT = 0, 1, 2, 3
SRDR_FLAG_CONSTRAINED, SRDR_FLAG_END_LOAD = 1, 2
SRDR_SWEEP_LAYOUT_3D, SRDR_SWEEP_LAYOUT_2D = 0, 1
SRDR_BATCH_AUTO, SRDR_BATCH_SHARED, SRDR_BATCH_STREAMS = 0, 1, 2
SRDR_FIELD_PB, SRDR_FIELD_B0 = 0, 1

# every symbol include/srdr.h declares
EXPORTS = [
    "srdr_body_create", "srdr_body_create_particles", "srdr_body_step", "srdr_body_relax",
    "srdr_body_read_displacement", "srdr_body_read_velocity", "srdr_body_write_state",
    "srdr_body_info", "srdr_body_stats", "srdr_body_read_neighbours", "srdr_body_read_cells",
    "srdr_body_read_field", "srdr_body_destroy", "srdr_last_error", "srdr_philox4x64_10",
    "srdr_random_phi", "srdr_body_profile", "srdr_body_kernel_times",
    "srdr_kinetic_energy_noalloc", "srdr_body_tune", "srdr_desc_particle_count",
    "srdr_body_pass_mapping", "srdr_body_sweep_sync", "srdr_body_sweep_lanes", "srdr_body_debug_stall_sweep",
    "srdr_batch_create", "srdr_batch_step", "srdr_batch_run", "srdr_batch_info", "srdr_batch_mode",
    "srdr_batch_destroy", "srdr_batch_relax", "srdr_server_create", "srdr_server_configure",
    "srdr_server_submit", "srdr_server_poll", "srdr_server_wait", "srdr_server_stats",
    "srdr_server_destroy",
]
KERNEL_CLASSES = ["pass_a", "pass_b", "sweep", "finish", "ke_final"]


class SrdrError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"srdr {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class srdr_body_desc(C.Structure):
    _fields_ = [
        ("dim", C.c_int),
        ("extent", C.c_double * 3),
        ("dp", C.c_double),
        ("clamp_axis", C.c_int),
        ("clamp_layers", C.c_int),
        ("presc_layers", C.c_int),
        ("presc_disp", C.c_double * 3),
        ("end_load_layer", C.c_int),
        ("material", C.c_int),
        ("rho0", C.c_double), ("E", C.c_double), ("nu", C.c_double),
        ("h_over_dp", C.c_double),
        ("gravity", C.c_double * 3),
        ("end_load", C.c_double * 3),
        ("beta", C.c_double), ("L_char", C.c_double), ("alpha", C.c_double),
        ("seed", C.c_uint64),
        ("damping", C.c_int),
        ("precision", C.c_int),
        ("dt", C.c_double),
        ("twist", C.c_double * 4),
        ("sweep_layout", C.c_int),
        ("pass_layout", C.c_int),
    ]


class srdr_stats(C.Structure):
    _fields_ = [("step", C.c_int64), ("damped_steps", C.c_int64), ("ke", C.c_double),
                ("ke_max", C.c_double), ("eta", C.c_double), ("dt", C.c_double),
                ("converged", C.c_int), ("launches", C.c_int64),
                ("sweep_cells_per_warp", C.c_int), ("pass_mapping", C.c_int),
                ("sweep_sync", C.c_int)]


class srdr_kernel_times(C.Structure):
    _fields_ = [("ms", C.c_double * 5), ("launches", C.c_int64 * 5), ("intervals", C.c_int64 * 5)]


_lib = None


def lib():
    """Load libsrdr.so (built by paper_2103_08932_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise OSError(f"{LIB_PATH} is missing: build it with "
                      "`python -m paper_2103_08932_gb300.build` (no CPU fallback exists)")
    L = C.CDLL(LIB_PATH)
    p, i64, d = C.c_void_p, C.c_int64, C.c_double
    st = C.c_int
    sig = {
        "srdr_body_create": (st, [C.POINTER(srdr_body_desc), p, C.POINTER(p)]),
        "srdr_body_create_particles": (st, [C.POINTER(srdr_body_desc), i64, p, p, p, p, p,
                                            C.POINTER(p)]),
        "srdr_body_step": (st, [p, i64]),
        "srdr_body_relax": (st, [p, d, i64, C.POINTER(i64), C.POINTER(d)]),
        "srdr_body_read_displacement": (st, [p, p, C.c_size_t]),
        "srdr_body_read_velocity": (st, [p, p, C.c_size_t]),
        "srdr_body_write_state": (st, [p, p, p, i64, d]),
        "srdr_body_info": (st, [p, C.POINTER(i64), C.POINTER(i64), C.POINTER(C.c_int),
                                C.POINTER(d)]),
        "srdr_body_stats": (st, [p, C.POINTER(srdr_stats)]),
        "srdr_body_read_neighbours": (st, [p, p, p]),
        "srdr_body_read_cells": (st, [p, p, p, p]),
        "srdr_body_read_field": (st, [p, C.c_int, p, C.c_size_t]),
        "srdr_body_destroy": (None, [p]),
        "srdr_last_error": (C.c_char_p, []),
        "srdr_philox4x64_10": (None, [p, p, p]),
        "srdr_random_phi": (d, [C.c_uint64, C.c_uint64]),
        "srdr_body_profile": (st, [p, C.c_int]),
        "srdr_body_kernel_times": (st, [p, C.POINTER(srdr_kernel_times)]),
        "srdr_body_tune": (st, [p, C.c_int, C.c_int]),
        "srdr_body_pass_mapping": (st, [p, C.c_int, C.c_int, C.c_int, C.c_int]),
        "srdr_body_sweep_lanes": (st, [p, C.c_int]),
        "srdr_body_sweep_sync": (st, [p, C.c_int]),
        "srdr_body_debug_stall_sweep": (st, [p]),
        "srdr_desc_particle_count": (st, [C.POINTER(srdr_body_desc), C.POINTER(i64)]),
        "srdr_batch_create": (st, [p, C.c_int, p, C.POINTER(p)]),
        "srdr_batch_step": (st, [p, i64]),
        "srdr_batch_run": (st, [p, d, i64, p, p]),
        "srdr_batch_info": (st, [p, C.POINTER(i64), C.POINTER(i64), C.POINTER(C.c_int),
                                 C.POINTER(C.c_int)]),
        "srdr_batch_destroy": (None, [p]),
        "srdr_batch_mode": (st, [p, C.c_int]),
        "srdr_batch_relax": (st, [p, C.c_int, d, i64, p, p]),
    }
    for name, (rt, args) in sig.items():
        f = getattr(L, name)
        f.restype = rt
        f.argtypes = args
    _lib = L
    return L


def last_error() -> str:
    return lib().srdr_last_error().decode(errors="replace")


def _check(status):
    if status != SRDR_OK:
        raise SrdrError(status, last_error())
    return status


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def make_desc(spec, precision=SRDR_FP64, damping=SRDR_DAMP_PARTICLE, dt=0.0,
              sweep_layout=0, pass_layout=0) -> srdr_body_desc:
    """C description from a synth.BodySpec-like object."""
    d = srdr_body_desc()
    d.dim = spec.dim
    ext = list(spec.extent) + [0.0] * (3 - len(spec.extent))
    d.extent = (C.c_double * 3)(*ext)
    d.dp = spec.dp
    d.clamp_axis = spec.clamp_axis
    d.clamp_layers = spec.clamp_layers
    d.presc_layers = spec.presc_layers
    d.presc_disp = (C.c_double * 3)(*spec.presc_disp)
    d.end_load_layer = 1 if spec.end_load_layer else 0
    d.material = spec.material
    d.rho0, d.E, d.nu = spec.rho0, spec.E, spec.nu
    d.h_over_dp = spec.h_over_dp
    d.gravity = (C.c_double * 3)(*spec.gravity)
    d.end_load = (C.c_double * 3)(*spec.end_load)
    d.beta, d.L_char, d.alpha = spec.beta, spec.L_char, spec.alpha
    d.seed = spec.seed
    d.damping = damping
    d.precision = precision
    d.dt = dt
    d.twist = (C.c_double * 4)(*getattr(spec, "twist", (0.0, 0.0, 0.0, 0.0)))
    d.sweep_layout = sweep_layout
    d.pass_layout = pass_layout
    return d


def _vec3(x):
    x = np.asarray(x, dtype=np.float64)
    if x.ndim == 2 and x.shape[1] != 3:
        y = np.zeros((x.shape[0], 3))
        y[:, : x.shape[1]] = x
        x = y
    return np.ascontiguousarray(x.reshape(-1, 3))


def srdr_body_create(desc: srdr_body_desc, stream: int = 0) -> int:
    h = C.c_void_p()
    _check(lib().srdr_body_create(C.byref(desc), C.c_void_p(stream), C.byref(h)))
    return h.value


def srdr_body_create_particles(desc, r0, vol=None, flags=None, u0=None, stream: int = 0) -> int:
    r = _vec3(r0)
    v = None if vol is None else np.ascontiguousarray(np.asarray(vol, dtype=np.float64))
    f = None if flags is None else np.ascontiguousarray(np.asarray(flags, dtype=np.uint8))
    u = None if u0 is None else _vec3(u0)
    h = C.c_void_p()
    _check(lib().srdr_body_create_particles(C.byref(desc), r.shape[0], _ptr(r), _ptr(v), _ptr(f),
                                            _ptr(u), C.c_void_p(stream), C.byref(h)))
    return h.value


class Body:
    """Owning handle of one device-resident body."""

    def __init__(self, desc: srdr_body_desc, r0=None, vol=None, flags=None, u0=None,
                 stream: int = 0):
        self.desc = desc
        if r0 is None:
            self.h = srdr_body_create(desc, stream)
        else:
            self.h = srdr_body_create_particles(desc, r0, vol, flags, u0, stream)
        n, nnz, nc, dt = C.c_int64(), C.c_int64(), C.c_int(), C.c_double()
        _check(lib().srdr_body_info(self.h, C.byref(n), C.byref(nnz), C.byref(nc), C.byref(dt)))
        self.n, self.nnz, self.ncells, self.dt = n.value, nnz.value, nc.value, dt.value

    def close(self):
        if getattr(self, "h", None):
            lib().srdr_body_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, nsteps=1):
        return _check(lib().srdr_body_step(self.h, int(nsteps)))

    def relax(self, ke_ratio=1e-8, max_steps=10**7, check=True):
        st, r = C.c_int64(), C.c_double()
        status = lib().srdr_body_relax(self.h, ke_ratio, int(max_steps), C.byref(st), C.byref(r))
        if check:
            _check(status)
        return status, st.value, r.value

    def displacement(self):
        out = np.zeros((self.n, 3))
        _check(lib().srdr_body_read_displacement(self.h, _ptr(out), out.size))
        return out

    def velocity(self):
        out = np.zeros((self.n, 3))
        _check(lib().srdr_body_read_velocity(self.h, _ptr(out), out.size))
        return out

    def write_state(self, u=None, v=None, step_index=0, ke_max=0.0):
        ua = None if u is None else _vec3(u)
        va = None if v is None else _vec3(v)
        _check(lib().srdr_body_write_state(self.h, _ptr(ua), _ptr(va), int(step_index), ke_max))

    def stats(self):
        s = srdr_stats()
        _check(lib().srdr_body_stats(self.h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in srdr_stats._fields_}

    def tune(self, sweep_cells_per_warp=0, sweep_warps_per_block=0):
        _check(lib().srdr_body_tune(self.h, int(sweep_cells_per_warp), int(sweep_warps_per_block)))

    def sweep_sync(self, mode=0):
        """SRDR_SWEEP_AUTO (0), SRDR_SWEEP_BARRIER (1) or SRDR_SWEEP_CELLS (2)."""
        _check(lib().srdr_body_sweep_sync(self.h, int(mode)))

    def sweep_lanes(self, lanes=0):
        """Width of the sweep's serial chain: 0 (autotuned), 16 or 32."""
        _check(lib().srdr_body_sweep_lanes(self.h, int(lanes)))

    def debug_stall_sweep(self):
        """Make every wait of the next damping sweep run out (failure-path test hook)."""
        _check(lib().srdr_body_debug_stall_sweep(self.h))

    def pass_mapping(self, mapping=0, brick=(0, 0, 0)):
        """SRDR_PASS_AUTO (0), SRDR_PASS_SELL (1), SRDR_PASS_BRICKS (2) or
        SRDR_PASS_STENCIL (3, lattice-stencil bodies only),
        with the brick size in cells (0 = default)."""
        bx, by, bz = (int(x) for x in brick)
        _check(lib().srdr_body_pass_mapping(self.h, int(mapping), bx, by, bz))

    def profile(self, enable=True):
        """True / k > 0: time every (k-th) step's kernels with CUDA events; False / 0: stop."""
        k = (1 if enable else 0) if isinstance(enable, bool) else int(enable)
        _check(lib().srdr_body_profile(self.h, k))

    def kernel_times(self):
        t = srdr_kernel_times()
        _check(lib().srdr_body_kernel_times(self.h, C.byref(t)))
        return {name: {"ms": t.ms[k], "launches": t.launches[k], "intervals": t.intervals[k]}
                for k, name in enumerate(KERNEL_CLASSES)}

    def neighbours(self):
        row = np.zeros(self.n + 1, dtype=np.int64)
        col = np.zeros(max(self.nnz, 1), dtype=np.int64)
        _check(lib().srdr_body_read_neighbours(self.h, _ptr(row), _ptr(col)))
        return row, col[: self.nnz]

    def cells(self):
        cell = np.zeros(self.n, dtype=np.int64)
        colour = np.zeros(self.n, dtype=np.int32)
        order = np.zeros(self.n, dtype=np.int64)
        _check(lib().srdr_body_read_cells(self.h, _ptr(cell), _ptr(colour), _ptr(order)))
        return cell, colour, order

    def field(self, which):
        out = np.zeros((self.n, 3, 3))
        _check(lib().srdr_body_read_field(self.h, which, _ptr(out), out.size))
        return out


def srdr_philox4x64_10(counter, key):
    c = np.ascontiguousarray(np.asarray(counter, dtype=np.uint64))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint64))
    out = np.zeros(4, dtype=np.uint64)
    lib().srdr_philox4x64_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def srdr_random_phi(seed, step):
    return lib().srdr_random_phi(seed, step)


class Batch:
    """Several bodies relaxed together (srdr_batch_*).  The bodies must
    outlive the batch."""

    def __init__(self, bodies, stream: int = 0):
        self.bodies = list(bodies)
        arr = (C.c_void_p * len(self.bodies))(*[b.h for b in self.bodies])
        h = C.c_void_p()
        _check(lib().srdr_batch_create(arr, len(self.bodies), C.c_void_p(stream), C.byref(h)))
        self.h = h.value

    def close(self):
        if getattr(self, "h", None):
            lib().srdr_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, nsteps=1):
        _check(lib().srdr_batch_step(self.h, int(nsteps)))

    def mode(self, mode=SRDR_BATCH_AUTO):
        """SRDR_BATCH_AUTO (0), SRDR_BATCH_SHARED (1) or SRDR_BATCH_STREAMS (2)."""
        _check(lib().srdr_batch_mode(self.h, int(mode)))

    def run(self, ke_ratio=1e-8, max_steps=10**6):
        nb = len(self.bodies)
        st = np.zeros(nb, dtype=np.int32)
        steps = np.zeros(nb, dtype=np.int64)
        status = lib().srdr_batch_run(self.h, ke_ratio, int(max_steps), _ptr(st), _ptr(steps))
        return status, st, steps

    def info(self):
        s, l, g, t = C.c_int64(), C.c_int64(), C.c_int(), C.c_int()
        _check(lib().srdr_batch_info(self.h, C.byref(s), C.byref(l), C.byref(g), C.byref(t)))
        return {"steps": s.value, "launches": l.value, "sweep_cells_per_warp": g.value,
                "pass_threads": t.value}


def srdr_desc_particle_count(desc) -> int:
    n = C.c_int64()
    _check(lib().srdr_desc_particle_count(C.byref(desc), C.byref(n)))
    return n.value


def srdr_batch_relax(descs, ke_ratio=1e-8, max_steps=10**6):
    """Build, relax and free a batch of lattice bodies; returns (status,
    per-body status, list of displacement arrays [n_b][3])."""
    nb = len(descs)
    arr = (srdr_body_desc * nb)(*descs)
    outs = [np.zeros((srdr_desc_particle_count(d), 3)) for d in descs]
    ptrs = (C.c_void_p * nb)(*[o.ctypes.data for o in outs])
    st = np.zeros(nb, dtype=np.int32)
    status = lib().srdr_batch_relax(arr, nb, ke_ratio, int(max_steps), ptrs, _ptr(st))
    return status, st, outs


class srdr_server_report(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("refused", C.c_int64),
                ("queued", C.c_int64), ("in_flight", C.c_int64), ("peak_concurrent", C.c_int),
                ("bytes_in_use", C.c_size_t), ("particle_steps", C.c_int64),
                ("p50_latency_s", C.c_double), ("p99_latency_s", C.c_double),
                ("solves_per_s", C.c_double), ("not_converged", C.c_int64),
                ("failed", C.c_int64)]


def _server_sigs(L):
    p, i64, d = C.c_void_p, C.c_int64, C.c_double
    for name, rt, args in [
        ("srdr_server_create", C.c_int, [C.c_size_t, p, C.POINTER(p)]),
        ("srdr_server_configure", C.c_int, [p, d, i64, C.c_int, i64, C.c_size_t]),
        ("srdr_server_submit", C.c_int, [p, C.POINTER(srdr_body_desc), C.POINTER(C.c_uint64)]),
        ("srdr_server_poll", C.c_int, [p, C.c_uint64, p, C.c_size_t, C.POINTER(d)]),
        ("srdr_server_wait", C.c_int, [p, C.c_uint64, d, p, C.c_size_t, C.POINTER(d),
                                       C.POINTER(i64)]),
        ("srdr_server_stats", C.c_int, [p, C.POINTER(srdr_server_report)]),
        ("srdr_server_destroy", None, [p]),
    ]:
        f = getattr(L, name)
        f.restype = rt
        f.argtypes = args


class Server:
    """Continuous-batching relaxation server (srdr_server_*)."""

    def __init__(self, device_mem_budget, stream: int = 0, ke_ratio=1e-8, max_steps=10**6,
                 max_bodies=256, chunk_steps=256, queue_capacity=4096):
        L = lib()
        _server_sigs(L)
        h = C.c_void_p()
        _check(L.srdr_server_create(int(device_mem_budget), C.c_void_p(stream), C.byref(h)))
        self.h = h.value
        _check(L.srdr_server_configure(self.h, ke_ratio, int(max_steps), int(max_bodies),
                                       int(chunk_steps), int(queue_capacity)))
        self.sizes = {}

    def close(self):
        if getattr(self, "h", None):
            lib().srdr_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, desc):
        t = C.c_uint64()
        st = lib().srdr_server_submit(self.h, C.byref(desc), C.byref(t))
        if st != SRDR_OK:
            return st, None
        self.sizes[t.value] = srdr_desc_particle_count(desc)
        return st, t.value

    def poll(self, ticket):
        out = np.zeros((self.sizes[ticket], 3))
        lat = C.c_double()
        st = lib().srdr_server_poll(self.h, ticket, _ptr(out), out.size, C.byref(lat))
        return st, (out if st in (SRDR_OK, SRDR_ERR_NOT_CONVERGED) else None), lat.value

    def wait(self, ticket, timeout_s=600.0):
        out = np.zeros((self.sizes[ticket], 3))
        lat, steps = C.c_double(), C.c_int64()
        st = lib().srdr_server_wait(self.h, ticket, timeout_s, _ptr(out), out.size, C.byref(lat),
                                    C.byref(steps))
        return st, (out if st in (SRDR_OK, SRDR_ERR_NOT_CONVERGED) else None), lat.value, steps.value

    def stats(self):
        r = srdr_server_report()
        _check(lib().srdr_server_stats(self.h, C.byref(r)))
        return {k: getattr(r, k) for k, _ in srdr_server_report._fields_}
