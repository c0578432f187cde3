"""Pins of the oracle's method steps: splitting cell-linked list (Sec. 3.4),
neighbour lists, kernel-corrected kinematics (Eqs. correction-matrix,
deformation-gradient, the dF/dt equation), the momentum sum
(Eq. evaluate-momentum) and the damping operator (Sec. 3.1, 3.2).

Each check is tied to something other than the oracle's own formulas: the
paper's worked example, brute force, exact linear-field consistency, exact
conservation laws, a library least-squares solve, and a matrix exponential of
the explicit viscous operator.
"""
import math
import os

import numpy as np
import pytest
from scipy import linalg

from oracle import oracle as O
from paper_2103_08932_gb300 import synth as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _params(spec, **kw):
    d = dict(dim=spec.dim, material=spec.material, rho0=spec.rho0, E=spec.E, nu=spec.nu,
             h=spec.h, gravity=spec.gravity, end_load=spec.end_load, beta=spec.beta,
             L_char=spec.L_char, alpha=spec.alpha, seed=spec.seed)
    d.update(kw)
    return O.Params(**d)


def _body(spec, jitter=0.0, seed=0, **kw):
    if jitter > 0:
        r0, flags, u0 = S.jittered(spec, jitter, seed)
    else:
        r0, flags, u0 = S.lattice(spec)
    b = O.OracleBody(_params(spec, **kw), r0[:, :spec.dim], vol_default=spec.vol, flags=flags,
                     u0=u0[:, :spec.dim])
    return b, r0, flags


def small3d(**kw):
    d = dict(dim=3, extent=(0.012, 0.006, 0.008), dp=1e-3, clamp_axis=0, clamp_layers=3)
    d.update(kw)
    return S.BodySpec(**d)


def small2d(**kw):
    d = dict(dim=2, extent=(0.03, 0.008, 0.0), dp=1e-3, clamp_axis=0, clamp_layers=3)
    d.update(kw)
    return S.BodySpec(**d)


# ------------------------------------------------------------------ splitting CLL
def test_splitting_cll_matches_paper_example():
    """Sec. 3.4: on a grid of 6 columns x 9 cells numbered column by column,
    block 1 = {1,4,7,28,31,34} and block 9 = {21,24,27,48,51,54}."""
    rows = {}
    for l in open(os.path.join(GOLDEN, "splitting_cll_blocks.txt")):
        if l.strip() and not l.startswith("#"):
            k, v = l.split(":")
            rows[int(k)] = sorted(int(x) for x in v.split())
    # one particle at the centre of every cell, unit cells
    pts, number = [], []
    for ix in range(6):
        for iy in range(9):
            pts.append([ix + 0.5, iy + 0.5])
            number.append(iy + 9 * ix + 1)
    cell, colour, nc, order = O.cells(2, np.array(pts), 1.0)
    assert list(nc[:2]) == [6, 9]
    number = np.array(number)
    for block, cells in rows.items():
        assert sorted(number[colour == block - 1].tolist()) == cells
    # nine blocks of six cells each
    assert sorted(np.bincount(colour).tolist()) == [6] * 9


@pytest.mark.parametrize("dim", [2, 3])
def test_same_colour_cells_have_disjoint_footprints(dim):
    rng = np.random.default_rng(3)
    pts = rng.uniform(0, 10.0, size=(4000, dim))
    cell, colour, nc, order = O.cells(dim, pts, 1.0)
    ncell = int(np.prod(nc[:dim]))
    ic = np.stack([cell % nc[0], (cell // nc[0]) % nc[1], cell // (nc[0] * nc[1])], axis=1)
    by_colour = {}
    for c, i3 in zip(colour, ic):
        by_colour.setdefault(int(c), set()).add(tuple(i3))
    assert len(by_colour) == 3 ** dim
    for c, cells in by_colour.items():
        cells = np.array(sorted(cells))
        # every pair of distinct same-colour cells is >= 3 apart on some axis,
        # so their 3^d neighbourhoods never overlap
        d = np.abs(cells[:, None, :] - cells[None, :, :]).max(axis=2)
        np.fill_diagonal(d, 99)
        assert d.min() >= 3


def test_canonical_order_is_sorted_permutation():
    b, r0, _ = _body(small3d(), jitter=0.2, seed=4)
    cell, colour, order = b.cells()
    assert sorted(order.tolist()) == list(range(b.n))
    keys = list(zip(colour[order], cell[order], order))
    assert keys == sorted(keys)


# ------------------------------------------------------------------ neighbours
@pytest.mark.parametrize("dim,jit", [(2, 0.0), (2, 0.3), (3, 0.0), (3, 0.35)])
def test_cll_neighbours_equal_brute_force(dim, jit):
    spec = small2d() if dim == 2 else small3d()
    b, r0, _ = _body(spec, jitter=jit, seed=9)
    row, col = b.neighbours()
    brow, bcol = O.neighbours_brute(dim, r0[:, :dim], 2 * spec.h)
    assert np.array_equal(row, brow)
    assert np.array_equal(col, bcol)


def test_lattice_neighbour_counts():
    # 0 < r < 2.6 dp on a square / cubic lattice: 20 in 2D, 80 in 3D
    b2, _, _ = _body(small2d(extent=(0.02, 0.02, 0), clamp_axis=-1))
    row, _ = b2.neighbours()
    assert np.bincount(np.diff(row)).argmax() <= 20 and np.diff(row).max() == 20
    b3, _, _ = _body(small3d(extent=(0.008, 0.008, 0.008), clamp_axis=-1))
    row, _ = b3.neighbours()
    assert np.diff(row).max() == 80
    assert (sum(1 for i in range(-3, 4) for j in range(-3, 4) for k in range(-3, 4)
                if 0 < i * i + j * j + k * k < 2.6 ** 2)) == 80


# ------------------------------------------------------------------ kinematics
@pytest.mark.parametrize("dim,jit", [(2, 0.0), (2, 0.3), (3, 0.0), (3, 0.3)])
def test_patch_linear_displacement_gives_exact_F(dim, jit):
    """u = A X gives F_i = I + A at EVERY particle, boundary included: the
    correction matrix B0 makes the gradient exact for linear fields."""
    spec = small2d() if dim == 2 else small3d()
    b, r0, _ = _body(spec, jitter=jit, seed=1)
    rng = np.random.default_rng(7)
    A = np.zeros((3, 3))
    A[:dim, :dim] = rng.normal(scale=0.05, size=(dim, dim))
    u = r0 @ A.T
    F = b.F_from_u(u)
    want = np.eye(3)
    want[dim:, dim:] = 0
    want = want + A
    assert np.abs(F - want[None]).max() < 1e-12
    # the rate form: v = A X gives dF/dt = A
    Fd = b.Fdot(u)
    assert np.abs(Fd - A[None]).max() < 1e-12


def test_rate_and_displacement_forms_agree():
    """Reading of Eq. timestep-1/-3: dF/dt is linear in v and the position
    update is the same trapezoid, so F^{n+1/2} = I + grad(u^{n+1/2})."""
    spec = small2d(gravity=(0.0, -9.81, 0.0), material=S.NEO_HOOKEAN)
    ba, _, _ = _body(spec, f_form=O.F_RATE)
    bb, _, _ = _body(spec, f_form=O.F_DISPLACEMENT)
    ba.step(300)
    bb.step(300)
    ua, ub = ba.u, bb.u
    va, vb = ba.v, bb.v
    assert ba.damped_steps == bb.damped_steps > 0
    assert np.abs(ua - ub).max() <= 1e-10 * np.abs(ua).max()
    assert np.abs(va - vb).max() <= 1e-9 * np.abs(va).max()


# ------------------------------------------------------------------ momentum sum
@pytest.mark.parametrize("dim", [2, 3])
def test_internal_forces_sum_to_zero(dim):
    """grad0_i W_ij = -grad0_j W_ji, so sum_i m_i (dv_i/dt - g) = 0 for any F."""
    spec = (small2d() if dim == 2 else small3d())
    b, r0, flags = _body(spec, jitter=0.25, seed=2, gravity=(0.3, -9.81, 0.2))
    rng = np.random.default_rng(8)
    F = np.tile(np.eye(3), (b.n, 1, 1))
    F[:, :dim, :dim] += rng.normal(scale=0.05, size=(b.n, dim, dim))
    if dim == 2:
        F[:, 2, 2] = 0
    a = b.acc(F)
    g = np.array([0.3, -9.81, 0.2])
    g[dim:] = 0
    m = spec.rho0 * spec.vol
    f = m * (a - g[None])
    assert np.abs(f.sum(axis=0)).max() <= 1e-12 * np.abs(f).sum()


def test_homogeneous_deformation_interior_is_force_free():
    """Under uniform F, particles whose neighbours all have full support feel
    only gravity (the discrete divergence of a constant stress vanishes)."""
    spec = S.BodySpec(dim=3, extent=(0.012, 0.012, 0.012), dp=1e-3, clamp_axis=-1,
                      gravity=(0.0, -9.81, 0.0))
    b, r0, _ = _body(spec)
    F = np.tile(np.eye(3) + np.array([[0.01, 0.002, 0], [0.001, -0.004, 0.003], [0, 0.002, 0.006]]),
                (b.n, 1, 1))
    a = b.acc(F)
    c = np.array(spec.extent) / 2
    inner = np.all(np.abs(r0 - c) < c - 4 * spec.h - 1e-12, axis=1)
    assert inner.sum() > 0
    assert np.abs(a[inner] - np.array([0, -9.81, 0])).max() < 1e-9
    # and the boundary particles do feel the stress
    assert np.abs(a[~inner] - np.array([0, -9.81, 0])).max() > 1.0


# ------------------------------------------------------------------ damping
def _damp_body(dim=3, **kw):
    spec = small3d(clamp_axis=-1) if dim == 3 else small2d(clamp_axis=-1)
    return _body(spec, jitter=0.2, seed=5, **kw)


def _B(b, i, eta, dt, r0, dim, spec_h, vol):
    row, col = b.neighbours()
    js = col[row[i]:row[i + 1]]
    r = np.linalg.norm(r0[i, :dim] - r0[js, :dim], axis=1)
    dW = np.array([O.kernel_dW(dim, spec_h, x) for x in r])
    return js, 2 * eta * vol * vol * dW / r * dt


@pytest.mark.parametrize("dim", [2, 3])
def test_local_update_gradient_descent_step(dim):
    """Eqs. implicit-equation .. learning-rate-solve: the chosen increments
    (dv_i, dv_1 .. dv_N) = k grad E_i are the minimum-norm solution of the one
    linear equation E_i = (sum B - m_i) dv_i - sum B_j dv_j; we compare dv_i
    with numpy's least-squares solve of that equation."""
    b, r0, _ = _damp_body(dim)
    spec_h = 1.3e-3
    vol = 1e-3 ** dim
    m = 1000.0 * vol
    rng = np.random.default_rng(4)
    v = np.zeros((b.n, 3))
    v[:, :dim] = rng.normal(size=(b.n, dim))
    eta, dt = 30.0, 2e-5
    for i in [0, b.n // 2, b.n - 1]:
        js, B = _B(b, i, eta, dt, r0, dim, spec_h, vol)
        out = b.local_update(i, eta, dt, v)
        for c in range(dim):
            Ei = -np.sum(B * (v[i, c] - v[js, c]))
            row = np.concatenate([[B.sum() - m], -B])[None, :]
            x, *_ = np.linalg.lstsq(row, np.array([Ei]), rcond=None)
            assert abs((out[i, c] - v[i, c]) - x[0]) <= 1e-12 * max(1.0, abs(x[0]))


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("scheme", [O.DAMP_PARTICLE, O.DAMP_PAIRWISE])
def test_damping_conserves_momentum_exactly(dim, scheme):
    b, r0, _ = _damp_body(dim, damping=scheme)
    rng = np.random.default_rng(6)
    v = np.zeros((b.n, 3))
    v[:, :dim] = rng.normal(size=(b.n, dim))
    b.set(O.V, v)
    p0 = v.sum(axis=0)
    b.damp(40.0, 1e-5)
    v1 = b.v
    assert np.abs(v1.sum(axis=0) - p0).max() <= 1e-12 * np.abs(v).sum()
    assert np.abs(v1 - v).max() > 1e-3  # it did something


@pytest.mark.parametrize("scheme", [O.DAMP_PARTICLE, O.DAMP_PAIRWISE])
def test_damping_leaves_uniform_velocity_unchanged(scheme):
    b, _, _ = _damp_body(3, damping=scheme)
    v = np.tile([0.3, -1.2, 0.5], (b.n, 1))
    b.set(O.V, v)
    b.damp(40.0, 1e-5)
    assert np.abs(b.v - v).max() < 1e-13


def test_damping_sweep_does_not_raise_kinetic_energy_in_stable_range():
    """At |sum_j B_j| / m_i <= ~10 each local update dissipates."""
    for dim in (2, 3):
        b, _, _ = _damp_body(dim)
        rng = np.random.default_rng(12)
        for trial in range(3):
            v = np.zeros((b.n, 3))
            v[:, :dim] = rng.normal(size=(b.n, dim))
            b.set(O.V, v)
            ke0 = np.sum(v * v)
            b.damp(20.0, 2e-5)
            ke1 = np.sum(b.v ** 2)
            assert ke1 < ke0


def _explicit_viscous_operator(b, r0, dim, h, vol, eta):
    """Eq. damping-term as a matrix: (dv_i/dt)^nu = 2 eta/m_i sum_j V_i V_j v_ij/r_ij dW/dr."""
    row, col = b.neighbours()
    n = b.n
    m = 1000.0 * vol
    L = np.zeros((n, n))
    for i in range(n):
        for k in range(row[i], row[i + 1]):
            j = col[k]
            r = np.linalg.norm(r0[i, :dim] - r0[j, :dim])
            c = 2 * eta / m * vol * vol * O.kernel_dW(dim, h, r) / r
            L[i, i] += c
            L[i, j] -= c
    return L


@pytest.mark.parametrize("scheme,factor", [(O.DAMP_PARTICLE, 2.0), (O.DAMP_PAIRWISE, 2.0)])
def test_damping_is_consistent_with_explicit_viscous_term(scheme, factor):
    """As dt -> 0 the split operator S_d^{dt} tends to exp(c dt L) of the
    explicit operator L of Eq. damping-term.  Each local operator D_i applies
    every pair (i, j) to both i and j, and every pair is met from both of its
    particles, so a forward plus backward sweep at dt/2 each gives c = 2."""
    dim, h = 2, 1.3e-3
    spec = S.BodySpec(dim=2, extent=(0.008, 0.006, 0), dp=1e-3, clamp_axis=-1)
    r0, flags, _ = S.jittered(spec, 0.2, 3)
    b = O.OracleBody(_params(spec, damping=scheme), r0[:, :2], vol_default=1e-6)
    vol = 1e-6
    L = _explicit_viscous_operator(b, r0, dim, h, vol, 1.0)
    rng = np.random.default_rng(1)
    v = np.zeros((b.n, 3))
    v[:, :2] = rng.normal(size=(b.n, 2))
    errs = []
    for dt in [4e-5, 2e-5, 1e-5]:
        b.set(O.V, v)
        b.damp(1.0, dt / 2)
        got = b.v[:, :2]
        want = linalg.expm(factor * dt * L) @ v[:, :2]
        step = np.abs(want - v[:, :2]).max()
        errs.append(np.abs(got - want).max() / step)
    # relative error of the increment shrinks with dt (first-order consistency)
    assert errs[0] < 0.2
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 0.6 * errs[0]




# ------------------------------------------------------------------ explicit comparator
@pytest.mark.parametrize("dim", [2, 3])
def test_explicit_viscous_term_conserves_momentum_and_rigid_motion(dim):
    """Eq. damping-term is antisymmetric in (i, j): sum_i m_i a_i = 0 for any
    velocity field, and a uniform velocity is not damped."""
    ext = (0.008, 0.006, 0.0) if dim == 2 else (0.006, 0.005, 0.004)
    spec = S.BodySpec(dim=dim, extent=ext, dp=1e-3, clamp_axis=-1)
    r0, flags, _ = S.jittered(spec, 0.2, 7)
    b = O.OracleBody(_params(spec), r0[:, :dim], vol_default=spec.vol)
    rng = np.random.default_rng(3)
    v = np.zeros((b.n, 3))
    v[:, :dim] = rng.normal(size=(b.n, dim))
    a = b.viscous_acc(2.0, v)
    m = spec.rho0 * spec.vol
    p = (m * a).sum(axis=0)
    assert np.abs(p).max() <= 1e-12 * (m * np.abs(a)).sum()
    u = np.zeros((b.n, 3))
    u[:, :dim] = rng.normal(size=dim)
    assert np.abs(b.viscous_acc(2.0, u)).max() <= 1e-12 * np.abs(a).max()


def test_explicit_viscous_term_is_half_the_sweep_rate():
    """The split sweep S_d at eta~ tends to exp(2 dt L) (Sec. 3.1, checked
    above), so its rate (S_d v - v) / dt tends to twice the explicit
    acceleration of Eq. damping-term at the same eta: this pins the explicit
    comparator's term against the implicit scheme's code path."""
    spec = S.BodySpec(dim=2, extent=(0.008, 0.006, 0), dp=1e-3, clamp_axis=-1)
    r0, flags, _ = S.jittered(spec, 0.2, 3)
    b = O.OracleBody(_params(spec), r0[:, :2], vol_default=1e-6)
    rng = np.random.default_rng(5)
    v = np.zeros((b.n, 3))
    v[:, :2] = rng.normal(size=(b.n, 2))
    want = 2.0 * b.viscous_acc(1.0, v)[:, :2]
    errs = []
    for dt in [4e-6, 2e-6, 1e-6]:
        b.set(O.V, v)
        b.damp(1.0, dt / 2)
        rate = (b.v[:, :2] - v[:, :2]) / dt
        errs.append(np.abs(rate - want).max() / np.abs(want).max())
    assert errs[0] < 0.05
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 0.6 * errs[0]


def test_explicit_time_step_limit():
    """Eq. viscous-criteria-o: with the explicit comparator dt is at most
    0.5 h^2 / (nu D), nu = eta / rho0 (here the binding limit)."""
    spec = S.BodySpec(dim=2, extent=(0.02, 0.01, 0), dp=1e-3, clamp_axis=0, clamp_layers=3,
                      E=2e6, nu=0.3, beta=5.0, L_char=0.01)
    r0, flags, _ = S.lattice(spec)
    b = O.OracleBody(_params(spec, damping=O.DAMP_EXPLICIT), r0[:, :2], vol_default=spec.vol,
                     flags=flags)
    eta = O.eta(spec.beta, spec.rho0, spec.E, spec.L_char)
    limit = 0.5 * spec.h ** 2 / (eta / spec.rho0 * 2)
    assert b.dt == pytest.approx(limit, rel=1e-14)
    split = O.OracleBody(_params(spec, damping=O.DAMP_PARTICLE), r0[:, :2], vol_default=spec.vol,
                         flags=flags)
    assert split.dt > 10 * b.dt


# ------------------------------------------------------------------ twisting body force
def test_twist_force_is_a_rotation_about_the_axis():
    """Reading R17 of Eq. rotation-body-force: the force is perpendicular to
    the radius from the axis (y_c, z_c), has no axial component, grows as
    sin(pi x / 2L) from zero at the clamped face to gamma0 r at x = L, and
    turns counter-clockwise about +x for gamma0 > 0."""
    p = O.Params(dim=3, twist=(50.0, 0.2, 0.01, 0.05))
    rng = np.random.default_rng(11)
    for _ in range(50):
        r = rng.uniform([0, 0, 0], [0.2, 0.02, 0.1])
        g = O.twist_force(p, r)
        rad = np.array([0.0, r[1] - 0.01, r[2] - 0.05])
        assert g[0] == 0.0
        assert abs(g @ rad) <= 1e-15 * np.linalg.norm(g) * np.linalg.norm(rad) + 1e-300
        gamma = 50.0 * np.sin(np.pi * r[0] / 0.4)
        assert np.linalg.norm(g) == pytest.approx(abs(gamma) * np.linalg.norm(rad), rel=1e-13)
        assert np.cross(rad, g)[0] == pytest.approx(gamma * (rad @ rad), rel=1e-12)
    assert np.abs(O.twist_force(p, [0.0, 0.0, 0.0])).max() == 0.0
    tip = O.twist_force(p, [0.2, 0.02, 0.05])
    assert tip[2] == pytest.approx(50.0 * 0.01, rel=1e-14)


def test_twist_force_drives_the_first_step():
    """A body at rest has no stress, so its first undamped step gives every
    free particle v = dt (g + g_t(r0_i)); the time step sees the largest
    body-force magnitude."""
    spec = S.BodySpec(dim=3, extent=(0.008, 0.004, 0.004), dp=1e-3, clamp_axis=0, clamp_layers=3,
                      gravity=(0.0, -9.81, 0.0))
    tw = (2000.0, 0.008, 0.002, 0.002)
    r0, flags, _ = S.lattice(spec)
    b = O.OracleBody(_params(spec, damping=O.DAMP_NONE, twist=tw), r0, vol_default=spec.vol,
                     flags=flags)
    plain = O.OracleBody(_params(spec, damping=O.DAMP_NONE), r0, vol_default=spec.vol, flags=flags)
    p = _params(spec, twist=tw)
    force = np.array([O.twist_force(p, r) for r in r0]) + np.array(spec.gravity)
    assert b.dt == plain.dt  # the acoustic limit binds at this load
    # a load large enough for the body-force limit to bind: the largest |g + g_t|
    big = (2e9, 0.008, 0.002, 0.002)
    pb = _params(spec, damping=O.DAMP_NONE, twist=big)
    fb = np.array([O.twist_force(pb, r) for r in r0]) + np.array(spec.gravity)
    bb = O.OracleBody(pb, r0, vol_default=spec.vol, flags=flags)
    assert bb.dt == pytest.approx(0.6 * np.sqrt(spec.h / np.linalg.norm(fb, axis=1).max()), rel=1e-14)
    b.step(1)
    free = (flags & O.FLAG_CONSTRAINED) == 0
    assert np.abs(b.v[free] - b.dt * force[free]).max() <= 1e-12 * np.abs(b.dt * force).max()
    assert np.abs(b.v[~free]).max() == 0.0
