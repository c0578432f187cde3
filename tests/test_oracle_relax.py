"""Relaxation-level pins of the oracle (Sec. 3, Sec. 4.1).

* the static tip deflection of a cantilever under a small gravity load tends
  to the Timoshenko beam solution as the resolution grows;
* the converged static state does not depend on the damping strength beta nor
  on the random-choice probability alpha (Sec. 3.3, Sec. 4.1);
* the pairwise scheme closed form (Eq. pairwise-solve) solves Eq. pairwise-eq.
"""
import math
from dataclasses import replace

import numpy as np
import pytest

from oracle import oracle as O
from paper_2103_08932_gb300 import synth as S


def _run(spec, tol=1e-10, max_steps=200000, **kw):
    r0, flags, u0 = S.lattice(spec)
    d = dict(dim=spec.dim, material=spec.material, rho0=spec.rho0, E=spec.E, nu=spec.nu,
             h=spec.h, gravity=spec.gravity, beta=spec.beta, L_char=spec.L_char,
             alpha=spec.alpha, seed=spec.seed)
    d.update(kw)
    b = O.OracleBody(O.Params(**d), r0[:, :spec.dim], vol_default=spec.vol, flags=flags)
    status, steps, ratio = b.relax(tol, max_steps)
    assert status == 0, (status, steps, ratio)
    return b, r0


def _timoshenko(E, nu, rho, g, L, H):
    # plane strain: E' = E / (1 - nu^2); shear correction 5/6
    Ep = E / (1 - nu * nu)
    G = E / (2 * (1 + nu))
    return 3 * rho * g * L ** 4 / (2 * Ep * H * H) + rho * g * L * L / (2 * (5.0 / 6.0) * G)


def test_cantilever_tip_tends_to_timoshenko():
    E, nu, rho, g, L, H = 2e6, 0.3, 1000.0, 9.81e-3, 0.1, 0.02
    want = _timoshenko(E, nu, rho, g, L, H)
    errs = []
    for ndp in (10, 20):
        dp = H / ndp
        spec = S.BodySpec(dim=2, extent=(L, H, 0), dp=dp, clamp_axis=0, clamp_layers=3,
                          material=S.SVK, rho0=rho, E=E, nu=nu, gravity=(0, -g, 0), beta=0.5,
                          L_char=H, alpha=0.2, seed=0)
        b, r0 = _run(spec)
        tip = r0[:, 0] > L - dp
        got = -b.u[tip, 1].mean()
        errs.append(abs(got / want - 1))
    assert errs[0] < 0.15
    assert errs[1] < 0.06
    assert errs[1] < 0.5 * errs[0]


def test_converged_state_independent_of_damping():
    base = S.BodySpec(dim=2, extent=(0.1, 0.02, 0), dp=0.002, clamp_axis=0, clamp_layers=3,
                      material=S.NEO_HOOKEAN, rho0=1000.0, E=2e6, nu=0.3,
                      gravity=(0, -9.81, 0), beta=0.5, L_char=0.02, alpha=0.2, seed=0)
    runs = []
    for beta, alpha in [(0.5, 0.2), (1.0, 0.2), (0.5, 0.5)]:
        b, r0 = _run(replace(base, beta=beta, alpha=alpha), tol=1e-13)
        runs.append(b.u)
    ref = runs[0]
    scale = np.abs(ref).max()
    for u in runs[1:]:
        assert np.abs(u - ref).max() <= 5e-4 * scale


def test_pairwise_closed_form_solves_pair_equation():
    """Three particles, each the other two's neighbour.  D_i of the pairwise
    scheme is the pair solves (i,j1), (i,j2), (i,j2), (i,j1) over dt/2 each;
    every pair solve must satisfy Eq. pairwise-eq, which we solve here with
    numpy.linalg.solve as a 2x2 implicit system per component."""
    dp, h = 1e-3, 1.3e-3
    r0 = np.array([[0.0, 0.0], [1.2e-3, 0.3e-3], [0.2e-3, 1.1e-3]])
    spec = S.BodySpec(dim=2, extent=(0.003, 0.003, 0), dp=dp, clamp_axis=-1)
    p = O.Params(dim=2, material=S.SVK, rho0=1000.0, E=2e6, nu=0.3, h=h, damping=O.DAMP_PAIRWISE)
    b = O.OracleBody(p, r0, vol_default=dp * dp)
    row, col = b.neighbours()
    assert list(np.diff(row)) == [2, 2, 2]
    m = 1000.0 * dp * dp
    eta, dt = 30.0, 4e-5
    rng = np.random.default_rng(0)
    v = np.zeros((3, 3))
    v[:, :2] = rng.normal(size=(3, 2))

    def pair(vv, i, j, dtp):
        r = np.linalg.norm(r0[i] - r0[j])
        B = 2 * eta * (dp * dp) ** 2 * O.kernel_dW(2, h, r) / r * dtp
        out = vv.copy()
        for c in range(2):
            vij = vv[i, c] - vv[j, c]
            # m_i dvi = B (vij + dvi - dvj);  m_j dvj = -B (vij + dvi - dvj)
            A = np.array([[m - B, B], [B, m - B]])
            rhs = np.array([B * vij, -B * vij])
            dvi, dvj = np.linalg.solve(A, rhs)
            out[i, c] += dvi
            out[j, c] += dvj
        return out

    i = 0
    js = col[row[i]:row[i + 1]]
    want = v.copy()
    for j in list(js) + list(js[::-1]):
        want = pair(want, i, j, dt / 2)
    got = b.local_update(i, eta, dt, v)
    assert np.abs(got - want).max() < 1e-13 * np.abs(v).max()


def test_explicit_and_split_damping_reach_the_same_state():
    """The explicit-viscosity comparator (Eq. damping-term under Eq.
    viscous-criteria-o) and the split random-choice scheme relax the same
    cantilever to the same static state; the explicit run needs a smaller
    time step."""
    base = S.BodySpec(dim=2, extent=(0.06, 0.02, 0), dp=0.002, clamp_axis=0, clamp_layers=3,
                      material=S.NEO_HOOKEAN, rho0=1000.0, E=2e6, nu=0.3,
                      gravity=(0, -9.81, 0), beta=0.5, L_char=0.02, alpha=0.2, seed=0)
    split, _ = _run(base, tol=1e-13)
    expl, _ = _run(base, tol=1e-12, damping=O.DAMP_EXPLICIT)
    assert expl.dt < split.dt
    scale = np.abs(split.u).max()
    assert np.abs(expl.u - split.u).max() <= 5e-4 * scale
