"""The 2^d-colour sweep layout (SRDR_SWEEP_LAYOUT_2D: the splitting
cell-linked list with cells of edge 2 r_c in 2^d colours) on the GPU against
the oracle's same layout (reading R18).

Cells, colours and the sweep order must be bit-exact; FP64 within 1e-9 per
step, damped steps included, for both damping schemes; FP32-mixed within the
stated 1e-5 per-step velocity bound over 100 steps; the sweep's two
synchronisations give the same bits; the stress and force passes do not
depend on the layout."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2103_08932_gb300 import srdr
from paper_2103_08932_gb300 import synth as S

pytestmark = pytest.mark.gpu

L2D = srdr.SRDR_SWEEP_LAYOUT_2D


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2103_08932_gb300 import build
    build.build()
    srdr.lib()


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def oracle_for(spec, parts=None, damping=O.DAMP_PARTICLE, layout=O.SWEEP_2D):
    r0, flags, u0 = parts if parts is not None else S.lattice(spec)
    p = O.Params(dim=spec.dim, material=spec.material, rho0=spec.rho0, E=spec.E, nu=spec.nu,
                 h=spec.h, gravity=spec.gravity, end_load=spec.end_load, beta=spec.beta,
                 L_char=spec.L_char, alpha=spec.alpha, seed=spec.seed, damping=damping,
                 sweep_layout=layout)
    return O.OracleBody(p, r0[:, :spec.dim], vol_default=spec.vol, flags=flags)


def gpu_for(spec, parts=None, precision=srdr.SRDR_FP64, damping=srdr.SRDR_DAMP_PARTICLE, layout=L2D,
            pass_layout=srdr.SRDR_PASS_LAYOUT_AUTO):
    d = srdr.make_desc(spec, precision=precision, damping=damping, sweep_layout=layout, pass_layout=pass_layout)
    if parts is None:
        return srdr.Body(d)
    r0, flags, u0 = parts
    return srdr.Body(d, r0=r0, flags=flags, u0=u0)


B3 = S.BodySpec(dim=3, extent=(0.024, 0.008, 0.012), dp=1e-3, clamp_axis=0, clamp_layers=3,
                material=S.NEO_HOOKEAN, gravity=(0.0, -9.81, 0.0), beta=0.2, L_char=0.008,
                alpha=0.5, seed=2)
B2 = S.BodySpec(dim=2, extent=(0.05, 0.01, 0.0), dp=1e-3, clamp_axis=0, clamp_layers=3,
                material=S.SVK, gravity=(0.0, -9.81, 0.0), beta=0.2, L_char=0.01, alpha=0.5, seed=0)


@pytest.mark.parametrize("spec,jit", [(B2, 0.0), (B2, 0.3), (B3, 0.0), (B3, 0.35)])
def test_layout_cells_colours_order_bit_exact(spec, jit):
    parts = S.jittered(spec, jit, 11) if jit > 0 else S.lattice(spec)
    ob = oracle_for(spec, parts)
    gb = gpu_for(spec, parts)
    oc, ocol, oorder = ob.cells()
    gc, gcol, gorder = gb.cells()
    assert np.array_equal(oc, gc)
    assert np.array_equal(ocol, gcol)
    assert np.array_equal(oorder, gorder)
    assert len(set(gcol.tolist())) == 2 ** spec.dim
    orow, ocolidx = ob.neighbours()
    grow, gcolidx = gb.neighbours()
    assert np.array_equal(orow, grow) and np.array_equal(ocolidx, gcolidx)


@pytest.mark.parametrize("spec", [B2, B3], ids=["2d", "3d"])
@pytest.mark.parametrize("damping", [srdr.SRDR_DAMP_PARTICLE, srdr.SRDR_DAMP_PAIRWISE],
                         ids=["particle", "pairwise"])
def test_layout_fp64_steps_match_oracle(spec, damping):
    ob = oracle_for(spec, damping=damping)
    gb = gpu_for(spec, damping=damping)
    worst = 0.0
    for _ in range(10):
        ob.step(1)
        gb.step(1)
        worst = max(worst, rel(gb.velocity(), ob.v), rel(gb.displacement(), ob.u))
    assert ob.damped_steps == gb.stats()["damped_steps"] > 0
    assert worst <= 1e-9


def test_layout_jittered_fp64_matches_oracle():
    parts = S.jittered(B3, 0.3, 5)
    ob = oracle_for(B3, parts)
    gb = gpu_for(B3, parts)
    ob.step(8)
    gb.step(8)
    assert ob.damped_steps > 0
    assert rel(gb.velocity(), ob.v) <= 1e-9


def test_layout_fp32_mixed_100_steps():
    spec = S.scaled(S.cantilever_plate_3d(), 0.3)
    ob = oracle_for(spec)
    gb = gpu_for(spec, precision=srdr.SRDR_FP32_MIXED)
    worst = 0.0
    for _ in range(100):
        ob.step(1)
        gb.step(1)
        worst = max(worst, rel(gb.velocity(), ob.v))
    assert ob.damped_steps == gb.stats()["damped_steps"] > 0
    assert worst <= 1e-5


@pytest.mark.parametrize("precision", [srdr.SRDR_FP64, srdr.SRDR_FP32_MIXED])
def test_layout_sync_modes_bitwise_equal(precision):
    spec = B3 if precision == srdr.SRDR_FP64 else S.scaled(S.cantilever_plate_3d(), 0.2)
    outs = []
    for mode in (srdr.SRDR_SWEEP_BARRIER, srdr.SRDR_SWEEP_CELLS, srdr.SRDR_SWEEP_AUTO):
        b = gpu_for(spec, precision=precision)
        b.sweep_sync(mode)
        b.step(14)
        b.step(64)
        assert b.stats()["damped_steps"] > 0
        outs.append((b.velocity(), b.displacement()))
    for v, u in outs[1:]:
        assert np.array_equal(v, outs[0][0]) and np.array_equal(u, outs[0][1])


def test_layout_changes_only_the_sweep():
    """Undamped steps (alpha = 0) are bitwise the same in both layouts up to
    the order of the particles' sums, which the passes keep: the stress and
    force passes do not depend on the sweep layout."""
    from dataclasses import replace
    spec = replace(B3, alpha=0.0)
    a = gpu_for(spec, layout=srdr.SRDR_SWEEP_LAYOUT_3D)
    b = gpu_for(spec)
    a.step(20)
    b.step(20)
    assert rel(b.velocity(), a.velocity()) <= 1e-12


def test_layout_refused_by_batches_and_bricks():
    a = gpu_for(B3, pass_layout=srdr.SRDR_PASS_LAYOUT_SELL)
    with pytest.raises(srdr.SrdrError) as e:
        srdr.Batch([a])
    assert e.value.status == srdr.SRDR_ERR_INVALID
    with pytest.raises(srdr.SrdrError) as e:
        a.pass_mapping(srdr.SRDR_PASS_BRICKS)
    assert e.value.status == srdr.SRDR_ERR_INVALID
    bad = srdr.make_desc(B3, sweep_layout=7)
    with pytest.raises(srdr.SrdrError) as e:
        srdr.Body(bad)
    assert e.value.status == srdr.SRDR_ERR_INVALID
