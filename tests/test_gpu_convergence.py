"""Parity at convergence and over long runs, GPU (C ABI) against the FP64
oracle.

Tolerance: 1e-4 relative maximum displacement error at convergence,
|u_gpu - u_oracle|_inf / |u_oracle|_inf, at the oracle's stopping step; the
FP64 GPU run must also stop at the same step as the oracle.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2103_08932_gb300 import srdr
from paper_2103_08932_gb300 import synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2103_08932_gb300 import build
    build.build()
    srdr.lib()


def oracle_for(spec, threads=0, **kw):
    r0, flags, u0 = S.lattice(spec)
    p = O.Params(dim=spec.dim, material=spec.material, rho0=spec.rho0, E=spec.E, nu=spec.nu,
                 h=spec.h, gravity=spec.gravity, end_load=spec.end_load, beta=spec.beta,
                 L_char=spec.L_char, alpha=spec.alpha, seed=spec.seed)
    for k, v in kw.items():
        setattr(p, k, v)
    has_u0 = np.abs(u0).max() > 0
    return O.OracleBody(p, r0[:, :spec.dim], vol_default=spec.vol, flags=flags,
                        u0=u0[:, :spec.dim] if has_u0 else None, threads=threads)


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("material", [S.SVK, S.NEO_HOOKEAN])
def test_cantilever_2d_relaxed_fp64_same_step_and_displacement(material):
    """2D cantilever under gravity (100 x 10 + 3 clamped columns, FP64, beta =
    alpha = 0.2, seed 0), relaxed until KE/KE_max < 1e-8."""
    spec = S.cantilever_2d(material)
    ob = oracle_for(spec)
    st_o, steps_o, _ = ob.relax(1e-8, 400000)
    gb = srdr.Body(srdr.make_desc(spec, precision=srdr.SRDR_FP64))
    st_g, steps_g, _ = gb.relax(1e-8, 400000)
    assert st_o == 0 and st_g == srdr.SRDR_OK
    assert steps_g == steps_o
    assert rel(gb.displacement(), ob.u) <= 1e-4
    assert rel(gb.displacement(), ob.u) <= 1e-9  # FP64 against FP64
    assert gb.stats()["damped_steps"] == ob.damped_steps


def test_cantilever_2d_fp32_mixed_at_oracle_step():
    spec = S.cantilever_2d(S.NEO_HOOKEAN)
    ob = oracle_for(spec)
    st_o, steps_o, _ = ob.relax(1e-8, 400000)
    gb = srdr.Body(srdr.make_desc(spec, precision=srdr.SRDR_FP32_MIXED))
    gb.step(steps_o)
    assert rel(gb.displacement(), ob.u) <= 1e-4


_ORACLE_RELAXED = {}


def oracle_relaxed(name, spec, **kw):
    """The oracle relaxed to KE/KE_max < 1e-8 (OpenMP build on every host
    core: the same bits as the serial build), cached per body."""
    if name not in _ORACLE_RELAXED:
        import os
        ob = oracle_for(spec, threads=os.cpu_count() or 1, **kw)
        st, steps, _ = ob.relax(1e-8, 400000)
        assert st == 0
        _ORACLE_RELAXED[name] = (steps, ob.u, ob.damped_steps)
    return _ORACLE_RELAXED[name]


RELAX3D = [("plate-x0.3", S.scaled(S.cantilever_plate_3d(), 0.3), {}),
           ("block-16mm", S.compression_block_3d(dp=1e-3, edge=0.016), {"f_form": O.F_DISPLACEMENT})]


@pytest.mark.parametrize("name,spec,kw", RELAX3D, ids=[c[0] for c in RELAX3D])
@pytest.mark.parametrize("precision", [srdr.SRDR_FP64, srdr.SRDR_FP32_MIXED])
def test_3d_relaxed_against_oracle(name, spec, kw, precision):
    """3D bodies relaxed to KE/KE_max < 1e-8: the plate scaled x0.3 (60 x 6 x
    30 + 3 clamped layers, 11,340 particles) and the compression block (16 mm
    cube at dp = 1 mm, 5,632 particles).  The GPU run converges; FP64 stops
    at the oracle's step; the displacement at the oracle's stopping step is
    within 1e-4 relative (1e-9 for FP64 against FP64)."""
    steps_o, u_o, damped_o = oracle_relaxed(name, spec, **kw)
    gb = srdr.Body(srdr.make_desc(spec, precision=precision))
    st, steps_g, _ = gb.relax(1e-8, 400000)
    assert st == srdr.SRDR_OK
    if precision == srdr.SRDR_FP64:
        assert steps_g == steps_o
        assert gb.stats()["damped_steps"] == damped_o
    else:
        assert abs(steps_g - steps_o) <= max(2, steps_o // 100)
    if steps_g != steps_o:
        gb = srdr.Body(srdr.make_desc(spec, precision=precision))
        gb.step(steps_o)
    err = rel(gb.displacement(), u_o)
    assert err <= 1e-4
    if precision == srdr.SRDR_FP64:
        assert err <= 1e-9


@pytest.mark.parametrize("spec", [S.scaled(S.cantilever_plate_3d(), 0.2),
                                  S.compression_block_3d(dp=1e-3, edge=0.012)],
                         ids=["plate-x0.2", "block-12mm"])
def test_3d_fp32_mixed_long_run(spec):
    """FP32-mixed (the plate's and the block's production precision) against
    the FP64 oracle over 300 steps including damped ones."""
    ob = oracle_for(spec, f_form=O.F_DISPLACEMENT)
    ob.step(300)
    gb = srdr.Body(srdr.make_desc(spec, precision=srdr.SRDR_FP32_MIXED))
    gb.step(300)
    assert ob.damped_steps > 0
    assert rel(gb.displacement(), ob.u) <= 1e-4
