"""ctypes wrapper of the FP64 CPU oracle (srdr_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product package.  It
imports nothing from the product package and the product imports nothing from
here.

Arrays crossing this wrapper are numpy float64 in ORIGINAL particle order,
vectors shaped (n, 3) and tensors (n, 3, 3) (the third row/column is zero in
2D).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "srdr_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libsrdr_oracle.so")
# the same source built with OpenMP (stress / force loops over particles, the
# cells of one colour of the damping sweep over threads): identical bits
_LIB_OMP = os.path.join(_HERE, "_build", "libsrdr_oracle_omp.so")

SVK, NEO_HOOKEAN = 0, 1
DAMP_NONE, DAMP_PARTICLE, DAMP_PAIRWISE, DAMP_EXPLICIT = 0, 1, 2, 3
F_RATE, F_DISPLACEMENT = 0, 1
SWEEP_3D, SWEEP_2D = 0, 1
FLAG_CONSTRAINED, FLAG_END_LOAD = 1, 2
U, V, F, PB, B0, ACC = 0, 1, 2, 3, 4, 5


def _build_one(out: str, extra, force: bool) -> str:
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(_SRC)
            and os.path.getmtime(out) >= os.path.getmtime(os.path.join(_HERE, "srdr_oracle.h"))):
        return out
    tmp = out + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
                           *extra, "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction) if it is out of date:
    the serial library and the OpenMP one."""
    _build_one(_LIB_OMP, ["-fopenmp"], force)
    return _build_one(_LIB, [], force)


class _Params(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("material", C.c_int),
        ("rho0", C.c_double), ("E", C.c_double), ("nu", C.c_double),
        ("h", C.c_double),
        ("gravity", C.c_double * 3), ("end_load", C.c_double * 3),
        ("beta", C.c_double), ("L_char", C.c_double),
        ("alpha", C.c_double), ("seed", C.c_uint64),
        ("damping", C.c_int), ("f_form", C.c_int),
        ("dt", C.c_double),
        ("twist", C.c_double * 4),
        ("sweep_layout", C.c_int),
    ]


_lib = None
_lib_omp = None


def lib(omp: bool = False):
    """The serial oracle library, or with omp=True its OpenMP build."""
    global _lib, _lib_omp
    if omp:
        if _lib_omp is None:
            build()
            _lib_omp = _declare(C.CDLL(_LIB_OMP))
        return _lib_omp
    if _lib is None:
        _lib = _declare(C.CDLL(build()))
    return _lib


def threads_available() -> int:
    """Threads the OpenMP build uses by default (the host's cores)."""
    return int(lib(True).ora_threads())


def _declare(L):
    if True:
        d, i64, p = C.c_double, C.c_int64, C.c_void_p
        L.ora_kernel_W.restype = d
        L.ora_kernel_W.argtypes = [C.c_int, d, d]
        L.ora_kernel_dW.restype = d
        L.ora_kernel_dW.argtypes = [C.c_int, d, d]
        L.ora_lame.argtypes = [d, d, p, p]
        L.ora_eta.restype = d
        L.ora_eta.argtypes = [d, d, d, d]
        L.ora_pk2.argtypes = [C.c_int, C.c_int, d, d, p, p]
        L.ora_nh_energy.restype = d
        L.ora_nh_energy.argtypes = [C.c_int, d, d, p]
        L.ora_philox4x64_10.argtypes = [p, p, p]
        L.ora_phi.restype = d
        L.ora_phi.argtypes = [C.c_uint64, C.c_uint64]
        L.ora_cells.argtypes = [C.c_int, i64, p, d, p, p, p, p]
        L.ora_cells_base.argtypes = [C.c_int, i64, p, d, C.c_int, p, p, p, p]
        L.ora_neighbours_brute.restype = i64
        L.ora_neighbours_brute.argtypes = [C.c_int, i64, p, d, p, p]
        L.ora_body_create.restype = p
        L.ora_body_create.argtypes = [C.POINTER(_Params), i64, p, p, d, p, p, C.c_char_p, C.c_int]
        L.ora_body_destroy.argtypes = [p]
        for name, rt in [("ora_body_n", i64), ("ora_body_nnz", i64), ("ora_body_dt", d),
                         ("ora_body_eta", d), ("ora_body_step_index", i64), ("ora_body_ke", d),
                         ("ora_body_ke_max", d), ("ora_body_damped_steps", i64)]:
            getattr(L, name).restype = rt
            getattr(L, name).argtypes = [p]
        L.ora_body_get.argtypes = [p, C.c_int, p]
        L.ora_body_set.argtypes = [p, C.c_int, p]
        L.ora_body_neighbours.argtypes = [p, p, p]
        L.ora_body_cells.argtypes = [p, p, p, p]
        L.ora_body_step.restype = C.c_int
        L.ora_body_step.argtypes = [p, i64]
        L.ora_body_relax.restype = C.c_int
        L.ora_body_relax.argtypes = [p, d, i64, p, p]
        L.ora_body_F_from_u.argtypes = [p, p, p]
        L.ora_body_Fdot.argtypes = [p, p, p]
        L.ora_body_acc.argtypes = [p, p, p]
        L.ora_body_damp.argtypes = [p, d, d]
        L.ora_body_viscous_acc.argtypes = [p, d, p, p]
        L.ora_twist_force.argtypes = [p, p, p]
        L.ora_body_local_update.argtypes = [p, i64, d, d, p]
        L.ora_set_threads.argtypes = [C.c_int]
        L.ora_threads.restype = C.c_int
    return L


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _vec3(x, dim):
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if x.ndim == 2 and x.shape[1] == dim and dim != 3:
        y = np.zeros((x.shape[0], 3))
        y[:, :dim] = x
        x = y
    return np.ascontiguousarray(x.reshape(-1, 3))


# ---------------------------------------------------------------- closed pieces
def kernel_W(dim, h, r):
    return lib().ora_kernel_W(dim, h, r)


def kernel_dW(dim, h, r):
    return lib().ora_kernel_dW(dim, h, r)


def lame(E, nu):
    lam, mu = C.c_double(), C.c_double()
    lib().ora_lame(E, nu, C.byref(lam), C.byref(mu))
    return lam.value, mu.value


def eta(beta, rho0, E, L):
    return lib().ora_eta(beta, rho0, E, L)


def pk2(dim, material, lam, mu, F):
    Fm = np.zeros(9)
    Fm.reshape(3, 3)[:dim, :dim] = np.asarray(F, dtype=np.float64)[:dim, :dim]
    S = np.zeros(9)
    lib().ora_pk2(dim, material, lam, mu, _ptr(Fm), _ptr(S))
    return S.reshape(3, 3)[:dim, :dim].copy()


def nh_energy(dim, lam, mu, F):
    Fm = np.zeros(9)
    Fm.reshape(3, 3)[:dim, :dim] = np.asarray(F, dtype=np.float64)[:dim, :dim]
    return lib().ora_nh_energy(dim, lam, mu, _ptr(Fm))


def philox4x64_10(counter, key):
    c = np.ascontiguousarray(np.asarray(counter, dtype=np.uint64))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint64))
    out = np.zeros(4, dtype=np.uint64)
    lib().ora_philox4x64_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def twist_force(params, r):
    """Rotational body force of reading R17 at reference position r."""
    ra = np.ascontiguousarray(np.asarray(r, dtype=np.float64).reshape(3))
    out = np.zeros(3)
    cp = params.to_c()
    lib().ora_twist_force(C.byref(cp), _ptr(ra), _ptr(out))
    return out


def phi(seed, step):
    return lib().ora_phi(seed, step)


def cells(dim, r0, rc, base=3):
    r = _vec3(r0, dim)
    n = r.shape[0]
    cell = np.zeros(n, dtype=np.int64)
    colour = np.zeros(n, dtype=np.int32)
    order = np.zeros(n, dtype=np.int64)
    nc = np.zeros(3, dtype=np.int64)
    if base == 3:
        lib().ora_cells(dim, n, _ptr(r), rc, _ptr(cell), _ptr(colour), _ptr(nc), _ptr(order))
    else:
        lib().ora_cells_base(dim, n, _ptr(r), rc, base, _ptr(cell), _ptr(colour), _ptr(nc), _ptr(order))
    return cell, colour, nc, order


def neighbours_brute(dim, r0, cutoff):
    r = _vec3(r0, dim)
    n = r.shape[0]
    nnz = lib().ora_neighbours_brute(dim, n, _ptr(r), cutoff, None, None)
    row = np.zeros(n + 1, dtype=np.int64)
    col = np.zeros(max(nnz, 1), dtype=np.int64)
    lib().ora_neighbours_brute(dim, n, _ptr(r), cutoff, _ptr(row), _ptr(col))
    return row, col[:nnz]


# ---------------------------------------------------------------- the body
@dataclass
class Params:
    dim: int = 3
    material: int = NEO_HOOKEAN
    rho0: float = 1000.0
    E: float = 2e6
    nu: float = 0.3
    h: float = 1.3e-3
    gravity: tuple = (0.0, -9.81, 0.0)
    end_load: tuple = (0.0, 0.0, 0.0)
    beta: float = 0.2
    L_char: float = 0.02
    alpha: float = 0.2
    seed: int = 0
    damping: int = DAMP_PARTICLE
    f_form: int = F_RATE
    dt: float = 0.0
    twist: tuple = (0.0, 0.0, 0.0, 0.0)  # (gamma0, L, y_c, z_c), reading R17
    sweep_layout: int = SWEEP_3D  # reading R18: SWEEP_2D = 2^d colours over cells of edge 4h

    def to_c(self) -> _Params:
        g = list(self.gravity) + [0.0] * (3 - len(self.gravity))
        e = list(self.end_load) + [0.0] * (3 - len(self.end_load))
        return _Params(self.dim, self.material, self.rho0, self.E, self.nu, self.h,
                       (C.c_double * 3)(*g), (C.c_double * 3)(*e), self.beta, self.L_char,
                       self.alpha, self.seed, self.damping, self.f_form, self.dt,
                       (C.c_double * 4)(*self.twist), self.sweep_layout)


class OracleBody:
    """An oracle body over arbitrary reference positions r0 (n, dim)."""

    def __init__(self, params: Params, r0, vol=None, vol_default=None, flags=None, u0=None,
                 threads: int = 0):
        """threads > 0: step on the OpenMP build with that many threads (the
        same bits as the serial build); 0: the serial build."""
        self._L = lib(True) if threads > 0 else lib()
        if threads > 0:
            self._L.ora_set_threads(int(threads))
        self.params = params
        dim = params.dim
        self.dim = dim
        r = _vec3(r0, dim)
        self.n = r.shape[0]
        self._keep = [r]
        vp = None
        if vol is not None:
            va = np.ascontiguousarray(np.asarray(vol, dtype=np.float64))
            self._keep.append(va)
            vp = _ptr(va)
        fp = None
        if flags is not None:
            fa = np.ascontiguousarray(np.asarray(flags, dtype=np.uint8))
            self._keep.append(fa)
            fp = _ptr(fa)
        up = None
        if u0 is not None:
            ua = _vec3(u0, dim)
            self._keep.append(ua)
            up = _ptr(ua)
        err = C.create_string_buffer(256)
        self._cp = params.to_c()
        vd = float(vol_default) if vol_default is not None else 0.0
        self._h = self._L.ora_body_create(C.byref(self._cp), self.n, _ptr(r), vp, vd, fp, up, err, 256)
        if not self._h:
            raise ValueError("oracle body: " + err.value.decode())

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.ora_body_destroy(h)
            self._h = None

    # scalars
    @property
    def nnz(self):
        return self._L.ora_body_nnz(self._h)

    @property
    def dt(self):
        return self._L.ora_body_dt(self._h)

    @property
    def eta(self):
        return self._L.ora_body_eta(self._h)

    @property
    def step_index(self):
        return self._L.ora_body_step_index(self._h)

    @property
    def ke(self):
        return self._L.ora_body_ke(self._h)

    @property
    def ke_max(self):
        return self._L.ora_body_ke_max(self._h)

    @property
    def damped_steps(self):
        return self._L.ora_body_damped_steps(self._h)

    # arrays
    def get(self, what):
        w = 3 if what in (U, V, ACC) else 9
        out = np.zeros((self.n, w))
        self._L.ora_body_get(self._h, what, _ptr(out))
        return out if w == 3 else out.reshape(self.n, 3, 3)

    def set(self, what, arr):
        a = np.ascontiguousarray(np.asarray(arr, dtype=np.float64).reshape(self.n, -1))
        if what in (U, V) and a.shape[1] != 3:
            a = _vec3(a, self.dim)
        self._L.ora_body_set(self._h, what, _ptr(a))

    @property
    def u(self):
        return self.get(U)

    @property
    def v(self):
        return self.get(V)

    def neighbours(self):
        row = np.zeros(self.n + 1, dtype=np.int64)
        col = np.zeros(max(self.nnz, 1), dtype=np.int64)
        self._L.ora_body_neighbours(self._h, _ptr(row), _ptr(col))
        return row, col[: self.nnz]

    def cells(self):
        cell = np.zeros(self.n, dtype=np.int64)
        colour = np.zeros(self.n, dtype=np.int32)
        order = np.zeros(self.n, dtype=np.int64)
        self._L.ora_body_cells(self._h, _ptr(cell), _ptr(colour), _ptr(order))
        return cell, colour, order

    def step(self, nsteps=1):
        return self._L.ora_body_step(self._h, nsteps)

    def relax(self, tol=1e-8, max_steps=10**7):
        st, ratio = C.c_int64(), C.c_double()
        status = self._L.ora_body_relax(self._h, tol, max_steps, C.byref(st), C.byref(ratio))
        return status, st.value, ratio.value

    def F_from_u(self, u):
        ua = _vec3(u, self.dim)
        out = np.zeros((self.n, 9))
        self._L.ora_body_F_from_u(self._h, _ptr(ua), _ptr(out))
        return out.reshape(self.n, 3, 3)

    def Fdot(self, v):
        va = _vec3(v, self.dim)
        out = np.zeros((self.n, 9))
        self._L.ora_body_Fdot(self._h, _ptr(va), _ptr(out))
        return out.reshape(self.n, 3, 3)

    def acc(self, F):
        Fa = np.ascontiguousarray(np.asarray(F, dtype=np.float64).reshape(self.n, 9))
        out = np.zeros((self.n, 3))
        self._L.ora_body_acc(self._h, _ptr(Fa), _ptr(out))
        return out

    def viscous_acc(self, eta, v):
        """Eq. damping-term for the velocity field v (explicit comparator)."""
        va = _vec3(v, self.dim)
        out = np.zeros((self.n, 3))
        self._L.ora_body_viscous_acc(self._h, eta, _ptr(va), _ptr(out))
        return out

    def damp(self, eta_tilde, dt_loc):
        self._L.ora_body_damp(self._h, eta_tilde, dt_loc)

    def local_update(self, i, eta_tilde, dt_loc, v):
        va = _vec3(v, self.dim).copy()
        self._L.ora_body_local_update(self._h, int(i), eta_tilde, dt_loc, _ptr(va))
        return va
