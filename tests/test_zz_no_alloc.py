"""srdr_kinetic_energy_noalloc: the allocation-free kinetic-energy reduction.

Callers that cannot allocate device memory (their own pool or arena owns it,
or their footprint is fixed once they run) compute the kinetic energy of
their own device velocity arrays with this entry point; its scratch is a
fixed static device array inside the library.  This file checks, through the
C ABI, that two calls in a row return the same kinetic energy as the
library's regular reduction (srdr_body_stats after a step), and that sizes
beyond the stated maximum are refused.  It is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2103_08932_gb300 import srdr
from paper_2103_08932_gb300 import synth as S

pytestmark = pytest.mark.gpu

MAX_N = 16384 * 256


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2103_08932_gb300 import build
    build.build()
    L = srdr.lib()
    f = L.srdr_kinetic_energy_noalloc
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_void_p, C.c_void_p]
    return L


def _ke_noalloc(L, v_soa, mass, flags, precision, out, stream=0):
    st = L.srdr_kinetic_energy_noalloc(C.c_void_p(v_soa.data_ptr()), C.c_void_p(mass.data_ptr()),
                                      C.c_void_p(flags.data_ptr()), v_soa.shape[1], precision,
                                      C.c_void_p(out.data_ptr()), C.c_void_p(stream))
    assert st == srdr.SRDR_OK, srdr.last_error()


# each particle's term has the same roundings as the library's reduction (FP32
# velocities and masses are passed in as the body holds them); only the order
# of the FP64 additions differs
@pytest.mark.parametrize("precision,tol", [(srdr.SRDR_FP64, 1e-12), (srdr.SRDR_FP32_MIXED, 1e-12)])
def test_noalloc_kinetic_energy_matches_body_reduction(L, precision, tol):
    import torch
    spec = S.BodySpec(dim=3, extent=(0.03, 0.008, 0.012), dp=1e-3, clamp_axis=0, clamp_layers=3,
                      material=S.NEO_HOOKEAN, gravity=(0.0, -9.81, 0.0), beta=0.2,
                      L_char=0.008, alpha=0.5, seed=4)
    body = srdr.Body(srdr.make_desc(spec, precision=precision))
    r0, flags, _ = S.lattice(spec)
    dt = torch.float64 if precision == srdr.SRDR_FP64 else torch.float32
    mass_t = torch.full((body.n,), spec.rho0 * spec.vol, dtype=dt, device="cuda")
    flags_t = torch.from_numpy(flags.astype(np.uint8)).cuda()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for call in range(2):
        body.step(3)
        ke_ref = body.stats()["ke"]
        v = body.velocity()  # original order, [n][3]
        v_soa = torch.from_numpy(np.ascontiguousarray(v.T)).to(device="cuda", dtype=dt)
        out.fill_(-1.0)
        _ke_noalloc(L, v_soa, mass_t, flags_t, precision, out)
        torch.cuda.synchronize()
        ke = float(out.item())
        assert ke_ref > 0
        assert abs(ke - ke_ref) <= tol * ke_ref, (call, ke, ke_ref)
    body.close()


def test_noalloc_rejects_sizes_beyond_maximum(L):
    st = L.srdr_kinetic_energy_noalloc(C.c_void_p(16), C.c_void_p(16), None, MAX_N + 1,
                                      srdr.SRDR_FP64, C.c_void_p(16), None)
    assert st == srdr.SRDR_ERR_INVALID
    assert "exceeds" in srdr.last_error()
