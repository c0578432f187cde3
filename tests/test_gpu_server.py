"""Served relaxation with continuous batching (srdr_server_*), on the GPU.

Requests arrive while others are running and are admitted as slots and the
device-memory budget free up; every result must be BITWISE the same as the
same body relaxed alone.  Faulty requests (a singular body, a diverging
damping setting) are injected on the host and must not disturb the others.
"""
import time
from dataclasses import replace

import numpy as np
import pytest

from paper_2103_08932_gb300 import srdr
from paper_2103_08932_gb300 import synth as S

pytestmark = pytest.mark.gpu

TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2103_08932_gb300 import build
    build.build()
    srdr.lib()


def specs():
    base = S.BodySpec(dim=3, extent=(0.016, 0.006, 0.006), dp=1e-3, clamp_axis=0,
                      material=S.NEO_HOOKEAN, E=2e6, nu=0.3, gravity=(0, -9.81, 0), beta=0.5,
                      L_char=0.006, alpha=0.2, seed=21)
    return [
        base,
        replace(base, extent=(0.01, 0.005, 0.008), E=1e6, seed=22, alpha=0.3),
        replace(base, extent=(0.02, 0.004, 0.005), material=S.SVK, seed=23),
        replace(base, extent=(0.008, 0.008, 0.008), E=5e6, seed=24, alpha=0.5),
        replace(base, extent=(0.012, 0.006, 0.004), nu=0.4, seed=25),
    ]


def alone(spec, precision=srdr.SRDR_FP64):
    b = srdr.Body(srdr.make_desc(spec, precision=precision))
    status, steps, _ = b.relax(TOL, 200000, check=False)
    return status, b.displacement(), steps


def test_server_results_equal_alone_under_continuous_batching():
    sp = specs()
    want = [alone(s) for s in sp]
    # budget for about two of these bodies at a time: later requests must wait
    # for a retirement to be admitted
    one = max(srdr.srdr_desc_particle_count(srdr.make_desc(s)) for s in sp)
    budget = int(2.5 * one * (400 + 80 * 48))
    srv = srdr.Server(budget, ke_ratio=TOL, max_steps=200000, max_bodies=3, chunk_steps=128)
    tickets = []
    for s in sp[:2]:
        st, t = srv.submit(srdr.make_desc(s))
        assert st == srdr.SRDR_OK
        tickets.append(t)
    time.sleep(0.05)  # these arrive while the first two are on the GPU
    for s in sp[2:]:
        st, t = srv.submit(srdr.make_desc(s))
        assert st == srdr.SRDR_OK
        tickets.append(t)
    for t, (status, u, steps) in zip(tickets, want):
        st, got, lat, nsteps = srv.wait(t, 600.0)
        assert st == status == srdr.SRDR_OK
        assert nsteps == steps
        assert np.array_equal(got, u)
        assert lat > 0
    rep = srv.stats()
    assert rep["completed"] == len(sp) and rep["in_flight"] == 0 and rep["queued"] == 0
    assert 2 <= rep["peak_concurrent"] <= 3
    assert 0 < rep["p50_latency_s"] <= rep["p99_latency_s"]
    assert rep["solves_per_s"] > 0
    srv.close()


def test_server_isolates_faulty_requests():
    sp = specs()[:2]
    want = [alone(s) for s in sp]
    srv = srdr.Server(8 << 30, ke_ratio=TOL, max_steps=200000, max_bodies=8, chunk_steps=128)
    bad_singular = replace(sp[0], extent=(0.01, 0.001, 0.01), seed=31)  # one layer thick
    # a time step 50x the acoustic limit: the explicit integration blows up
    auto_dt = srdr.Body(srdr.make_desc(sp[0])).dt
    descs = [srdr.make_desc(sp[0]), srdr.make_desc(bad_singular),
             srdr.make_desc(sp[0], dt=50.0 * auto_dt), srdr.make_desc(sp[1])]
    tickets = [srv.submit(d)[1] for d in descs]
    res = [srv.wait(t, 600.0) for t in tickets]
    assert res[1][0] == srdr.SRDR_ERR_INVALID
    assert res[2][0] == srdr.SRDR_ERR_NONFINITE
    for (st, got, _, steps), (wst, u, wsteps) in zip([res[0], res[3]], want):
        assert st == wst == srdr.SRDR_OK
        assert steps == wsteps
        assert np.array_equal(got, u)
    rep = srv.stats()
    # only the two converged requests are solves; the faulty ones are counted apart
    assert rep["completed"] == 2 and rep["failed"] == 2 and rep["not_converged"] == 0
    srv.close()


def test_server_step_capped_request_is_not_a_solve():
    """A request retired at max_steps before its KE criterion is reported as
    SRDR_ERR_NOT_CONVERGED and counted apart: it adds nothing to the solves,
    the solves per second or the latency percentiles."""
    sp = specs()[0]
    srv = srdr.Server(8 << 30, ke_ratio=TOL, max_steps=128, max_bodies=4, chunk_steps=64)
    st, t = srv.submit(srdr.make_desc(sp))
    assert st == srdr.SRDR_OK
    st, _, _, steps = srv.wait(t, 600.0)
    assert st == srdr.SRDR_ERR_NOT_CONVERGED and steps == 128
    rep = srv.stats()
    assert rep["completed"] == 0 and rep["not_converged"] == 1 and rep["failed"] == 0
    assert rep["solves_per_s"] == 0.0
    assert rep["p50_latency_s"] == 0.0 and rep["p99_latency_s"] == 0.0
    srv.close()


def test_served_results_match_oracle():
    """Two requests served together (FP64) against the FP64 oracle relaxing
    each body alone to the same criterion: the same stopping step and the
    same displacement within rounding (and within the 1e-4 bar)."""
    from oracle import oracle as O
    sp = specs()[:2]
    want = []
    for s in sp:
        r0, flags, _ = S.lattice(s)
        p = O.Params(dim=3, material=s.material, rho0=s.rho0, E=s.E, nu=s.nu, h=s.h,
                     gravity=s.gravity, beta=s.beta, L_char=s.L_char, alpha=s.alpha, seed=s.seed)
        ob = O.OracleBody(p, r0, vol_default=s.vol, flags=flags)
        st, steps, _ = ob.relax(TOL, 200000)
        assert st == 0
        want.append((steps, ob.u))
    srv = srdr.Server(8 << 30, ke_ratio=TOL, max_steps=200000, max_bodies=4, chunk_steps=128)
    tickets = [srv.submit(srdr.make_desc(s))[1] for s in sp]
    for t, (steps, u) in zip(tickets, want):
        st, got, _, nsteps = srv.wait(t, 600.0)
        assert st == srdr.SRDR_OK and nsteps == steps
        err = np.abs(got - u).max() / np.abs(u).max()
        assert err <= 1e-4
        assert err <= 1e-9  # FP64 against FP64
    srv.close()


def test_server_refusals():
    sp = specs()[0]
    srv = srdr.Server(1 << 20, ke_ratio=TOL)  # 1 MiB: no body fits
    st, t = srv.submit(srdr.make_desc(sp))
    assert st == srdr.SRDR_ERR_NO_MEMORY and t is None
    srv.close()
    big = S.cantilever_plate_3d()  # runs for a long time at this tolerance
    srv = srdr.Server(8 << 30, ke_ratio=1e-14, max_steps=10**6, max_bodies=1, queue_capacity=1)
    st1, t1 = srv.submit(srdr.make_desc(big, precision=srdr.SRDR_FP32_MIXED))
    deadline = time.time() + 60
    while srv.stats()["in_flight"] == 0 and time.time() < deadline:
        time.sleep(0.01)
    st2, t2 = srv.submit(srdr.make_desc(sp))  # waits in the queue (no free slot)
    st3, t3 = srv.submit(srdr.make_desc(sp))  # queue full
    assert st1 == st2 == srdr.SRDR_OK
    assert st3 == srdr.SRDR_ERR_BUSY
    assert srv.poll(t1)[0] == srdr.SRDR_ERR_BUSY
    srv.close()  # drops the unfinished requests
