"""Batched relaxation (one set of launches for many bodies of uneven sizes)
against the same bodies relaxed one at a time through the C ABI.

Every body keeps its own arithmetic and reduction order inside a batch, so
the results must be BITWISE equal to the single-body runs, including the
step at which each body meets its own kinetic-energy criterion."""
import numpy as np
import pytest

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


def uneven_specs(dim=3):
    if dim == 2:
        return [
            S.BodySpec(dim=2, extent=(0.04, 0.008, 0), dp=1e-3, clamp_axis=0, material=S.SVK,
                       E=2e6, nu=0.3, gravity=(0, -9.81, 0), beta=0.5, L_char=0.008, alpha=0.2, seed=5),
            S.BodySpec(dim=2, extent=(0.02, 0.006, 0), dp=1e-3, clamp_axis=0, material=S.NEO_HOOKEAN,
                       E=1e6, nu=0.4, gravity=(0, -9.81, 0), beta=0.5, L_char=0.006, alpha=0.3, seed=6),
        ]
    return [
        S.BodySpec(dim=3, extent=(0.02, 0.006, 0.006), dp=1e-3, clamp_axis=0, material=S.NEO_HOOKEAN,
                   E=2e6, nu=0.3, gravity=(0, -9.81, 0), beta=0.5, L_char=0.006, alpha=0.2, seed=11),
        S.BodySpec(dim=3, extent=(0.012, 0.008, 0.01), dp=1e-3, clamp_axis=0, material=S.SVK,
                   E=5e5, nu=0.4, gravity=(0, 0, 0), end_load=(0, -30.0, 0), end_load_layer=True,
                   beta=0.5, L_char=0.008, alpha=0.3, seed=12),
        S.BodySpec(dim=3, extent=(0.008, 0.005, 0.005), dp=1e-3, clamp_axis=0, material=S.NEO_HOOKEAN,
                   E=5e6, nu=0.25, gravity=(0, -9.81, 0), beta=0.5, L_char=0.005, alpha=0.5, seed=13),
    ]


MODES = [srdr.SRDR_BATCH_SHARED, srdr.SRDR_BATCH_STREAMS]


def layout_for(mode):
    """Shared launches take sliced-ELL bodies; concurrent streams take any
    body (the lattice bodies here take the stencil)."""
    return srdr.SRDR_PASS_LAYOUT_SELL if mode == srdr.SRDR_BATCH_SHARED else srdr.SRDR_PASS_LAYOUT_AUTO


@pytest.mark.parametrize("mode", MODES, ids=["shared", "streams"])
@pytest.mark.parametrize("dim,precision,sync", [
    (3, srdr.SRDR_FP64, srdr.SRDR_SWEEP_AUTO), (3, srdr.SRDR_FP32_MIXED, srdr.SRDR_SWEEP_AUTO),
    (2, srdr.SRDR_FP64, srdr.SRDR_SWEEP_AUTO), (3, srdr.SRDR_FP32_MIXED, srdr.SRDR_SWEEP_CELLS),
    (3, srdr.SRDR_FP64, srdr.SRDR_SWEEP_BARRIER), (2, srdr.SRDR_FP32_MIXED, srdr.SRDR_SWEEP_CELLS)])
def test_batch_steps_equal_single_bodies(dim, precision, sync, mode):
    """Batched steps (shared launches with a barrier or cell-wise batched
    sweep, or every body on its own stream) equal the same bodies stepped
    alone (cell-wise or barrier single-body sweep) bit for bit; the bodies
    then keep stepping alone and still agree."""
    specs = uneven_specs(dim)
    lay = layout_for(mode)
    single = [srdr.Body(srdr.make_desc(s, precision=precision, pass_layout=lay)) for s in specs]
    for b in single:
        b.sweep_sync(srdr.SRDR_SWEEP_BARRIER if sync == srdr.SRDR_SWEEP_CELLS else srdr.SRDR_SWEEP_CELLS)
        b.step(40)
    bodies = [srdr.Body(srdr.make_desc(s, precision=precision, pass_layout=lay)) for s in specs]
    for b in bodies:
        b.sweep_sync(sync)
    batch = srdr.Batch(bodies)
    batch.mode(mode)
    batch.step(40)
    info = batch.info()
    assert info["sweep_cells_per_warp"] in (1, 2, 4) and info["pass_threads"] in (128, 256, 512)
    batch.close()
    for a, b in zip(single, bodies):
        a.step(25)
        b.step(25)  # alone after the batch: the cell-wise counts carry over
    for a, b in zip(single, bodies):
        assert np.array_equal(a.velocity(), b.velocity())
        assert np.array_equal(a.displacement(), b.displacement())
        sa, sb = a.stats(), b.stats()
        assert sa["damped_steps"] == sb["damped_steps"] > 0
        assert sa["ke"] == sb["ke"]


@pytest.mark.parametrize("mode", MODES, ids=["shared", "streams"])
def test_batch_relax_retires_each_body_at_its_own_step(mode):
    specs = uneven_specs(3)
    tol = 1e-6
    single_steps, single_u = [], []
    lay = layout_for(mode)
    for s in specs:
        b = srdr.Body(srdr.make_desc(s, pass_layout=lay))
        status, steps, ratio = b.relax(tol, 200000)
        single_steps.append(steps)
        single_u.append(b.displacement())
    bodies = [srdr.Body(srdr.make_desc(s, pass_layout=lay)) for s in specs]
    batch = srdr.Batch(bodies)
    batch.mode(mode)
    status, st, steps = batch.run(tol, 200000)
    assert status == srdr.SRDR_OK and list(st) == [0] * len(specs)
    assert list(steps) == single_steps
    assert len(set(single_steps)) > 1  # the bodies really retire at different steps
    for b, u in zip(bodies, single_u):
        assert np.array_equal(b.displacement(), u)
        assert b.stats()["converged"] == 1
    batch.close()


def test_batch_relax_one_call():
    specs = uneven_specs(3)[:2]
    descs = [srdr.make_desc(s) for s in specs]
    status, st, outs = srdr.srdr_batch_relax(descs, 1e-6, 200000)
    assert status == srdr.SRDR_OK and list(st) == [0, 0]
    for s, u in zip(specs, outs):
        b = srdr.Body(srdr.make_desc(s))
        b.relax(1e-6, 200000)
        assert np.array_equal(b.displacement(), u)


@pytest.mark.parametrize("mode", MODES, ids=["shared", "streams"])
def test_batch_step_cap_reports_not_converged(mode):
    specs = uneven_specs(3)[:1]
    bodies = [srdr.Body(srdr.make_desc(s, pass_layout=layout_for(mode))) for s in specs]
    batch = srdr.Batch(bodies)
    batch.mode(mode)
    status, st, steps = batch.run(1e-12, 50)
    assert status == srdr.SRDR_ERR_NOT_CONVERGED
    assert list(st) == [srdr.SRDR_ERR_NOT_CONVERGED] and list(steps) == [50]


def _oracle(spec):
    from oracle import oracle as O
    r0, flags, u0 = S.lattice(spec)
    p = O.Params(dim=spec.dim, material=spec.material, rho0=spec.rho0, E=spec.E, nu=spec.nu,
                 h=spec.h, gravity=spec.gravity, end_load=spec.end_load, beta=spec.beta,
                 L_char=spec.L_char, alpha=spec.alpha, seed=spec.seed)
    return O.OracleBody(p, r0[:, :spec.dim], vol_default=spec.vol, flags=flags)


@pytest.mark.parametrize("precision", [srdr.SRDR_FP64, srdr.SRDR_FP32_MIXED])
def test_batched_bodies_at_convergence_match_oracle(precision):
    """Two uneven bodies relaxed together as one batch against the FP64 oracle
    relaxing each of them alone (KE/KE_max < 1e-6): FP64 stops at the
    oracle's step within rounding; FP32-mixed is compared at the oracle's
    stopping step, within 1e-4 relative max displacement."""
    specs = uneven_specs(3)[:2]
    tol = 1e-6
    want = []
    for s in specs:
        ob = _oracle(s)
        st, steps, _ = ob.relax(tol, 200000)
        assert st == 0
        want.append((steps, ob.u, ob.damped_steps))
    bodies = [srdr.Body(srdr.make_desc(s, precision=precision)) for s in specs]
    batch = srdr.Batch(bodies)
    if precision == srdr.SRDR_FP64:
        status, st, steps = batch.run(tol, 200000)
        assert status == srdr.SRDR_OK
        assert list(steps) == [w[0] for w in want]
    else:
        # step the batch to each oracle stopping step in turn
        order = sorted(range(len(specs)), key=lambda k: want[k][0])
        done = 0
        got = [None] * len(specs)
        for k in order:
            batch.step(want[k][0] - done)
            done = want[k][0]
            got[k] = bodies[k].displacement()
    for k, (b, (steps, u, damped)) in enumerate(zip(bodies, want)):
        ug = b.displacement() if precision == srdr.SRDR_FP64 else got[k]
        err = np.abs(ug - u).max() / np.abs(u).max()
        assert err <= 1e-4
        if precision == srdr.SRDR_FP64:
            assert err <= 1e-9
            assert b.stats()["damped_steps"] == damped
    batch.close()


def test_batch_mode_rejects_unknown():
    b = srdr.Body(srdr.make_desc(uneven_specs(3)[0]))
    batch = srdr.Batch([b])
    with pytest.raises(srdr.SrdrError) as e:
        batch.mode(5)
    assert e.value.status == srdr.SRDR_ERR_INVALID


def test_shared_launches_take_sliced_ell_bodies_only():
    """A batch holding a lattice-stencil body refuses shared launches and
    keeps its mode; the same bodies created with the sliced ELL accept them."""
    spec = uneven_specs(3)[0]
    st = srdr.Body(srdr.make_desc(spec))
    assert st.stats()["pass_mapping"] == srdr.SRDR_PASS_STENCIL
    batch = srdr.Batch([st])
    with pytest.raises(srdr.SrdrError) as e:
        batch.mode(srdr.SRDR_BATCH_SHARED)
    assert e.value.status == srdr.SRDR_ERR_INVALID and "sliced-ELL" in srdr.last_error()
    batch.mode(srdr.SRDR_BATCH_STREAMS)
    batch.step(3)
    batch.close()
    sell = srdr.Body(srdr.make_desc(spec, pass_layout=srdr.SRDR_PASS_LAYOUT_SELL))
    batch = srdr.Batch([sell])
    batch.mode(srdr.SRDR_BATCH_SHARED)
    batch.step(3)
    batch.close()
