"""The 2^d-colour sweep layout of the oracle (reading R18: the splitting
cell-linked list with cells of edge 2 r_c = 4h, colour sum_a (i_a mod 2) 2^a).

Pins that do not use the oracle's own sweep formulas:
* geometry: every particle is touched (as the updated particle or as one of its
  neighbours) by at most one cell of each colour, on lattice and jittered
  particle sets, so the cells of a colour commute (brute force over the
  neighbour lists);
* the colour map against the definition written out independently (cell
  coordinates of edge 4h, parity per axis);
* the sweep conserves momentum exactly and leaves a uniform velocity alone,
  like the paper's layout;
* running the cells of one colour on several threads gives the serial bits;
* relaxed with either layout, a body reaches the same static state (the sweep
  order only changes the path to equilibrium).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2103_08932_gb300 import synth as S


def _params(spec, **kw):
    d = dict(dim=spec.dim, material=spec.material, rho0=spec.rho0, E=spec.E, nu=spec.nu,
             h=spec.h, gravity=spec.gravity, end_load=spec.end_load, beta=spec.beta,
             L_char=spec.L_char, alpha=spec.alpha, seed=spec.seed)
    d.update(kw)
    return O.Params(**d)


def _body(spec, jitter=0.0, seed=0, threads=0, **kw):
    r0, flags, u0 = S.jittered(spec, jitter, seed) if jitter > 0 else S.lattice(spec)
    b = O.OracleBody(_params(spec, **kw), r0[:, :spec.dim], vol_default=spec.vol, flags=flags,
                     threads=threads)
    return b, r0


def _spec(dim):
    if dim == 3:
        return S.BodySpec(dim=3, extent=(0.024, 0.012, 0.016), dp=1e-3, clamp_axis=-1)
    return S.BodySpec(dim=2, extent=(0.05, 0.02, 0.0), dp=1e-3, clamp_axis=-1)


@pytest.mark.parametrize("dim,jit", [(2, 0.0), (2, 0.35), (3, 0.0), (3, 0.35)])
def test_each_particle_is_touched_by_one_cell_per_colour(dim, jit):
    b, r0 = _body(_spec(dim), jitter=jit, seed=7, sweep_layout=O.SWEEP_2D)
    cell, colour, order = b.cells()
    row, col = b.neighbours()
    assert len(set(colour.tolist())) == 2 ** dim
    touched = [dict() for _ in range(b.n)]  # particle -> {colour: set of cells}
    for i in range(b.n):
        for j in [i] + col[row[i]:row[i + 1]].tolist():
            touched[j].setdefault(int(colour[i]), set()).add(int(cell[i]))
    assert all(len(cs) == 1 for t in touched for cs in t.values())


@pytest.mark.parametrize("dim", [2, 3])
def test_colour_map_is_parity_of_cells_of_edge_4h(dim):
    spec = _spec(dim)
    b, r0 = _body(spec, jitter=0.3, seed=3, sweep_layout=O.SWEEP_2D)
    cell, colour, order = b.cells()
    edge = 4.0 * spec.h
    lo = r0[:, :dim].min(axis=0)
    n_ax = np.floor((r0[:, :dim].max(axis=0) - lo) / edge).astype(int) + 1
    ic = np.clip(np.floor((r0[:, :dim] - lo) / edge).astype(int), 0, n_ax - 1)
    want_colour = sum((ic[:, a] % 2) * 2 ** a for a in range(dim))
    assert np.array_equal(colour, want_colour)
    want_cell = ic[:, 0] + n_ax[0] * (ic[:, 1] + (n_ax[1] * ic[:, 2] if dim == 3 else 0))
    assert np.array_equal(cell, want_cell)
    keys = list(zip(colour[order], cell[order], order))
    assert keys == sorted(keys)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("scheme", [O.DAMP_PARTICLE, O.DAMP_PAIRWISE])
def test_sweep_with_2d_layout_conserves_momentum(dim, scheme):
    b, r0 = _body(_spec(dim), jitter=0.2, seed=5, damping=scheme, sweep_layout=O.SWEEP_2D)
    rng = np.random.default_rng(6)
    v = np.zeros((b.n, 3))
    v[:, :dim] = rng.normal(size=(b.n, dim))
    b.set(O.V, v)
    b.damp(40.0, 1e-5)
    v1 = b.v
    assert np.abs(v1.sum(axis=0) - v.sum(axis=0)).max() <= 1e-12 * np.abs(v).sum()
    assert np.abs(v1 - v).max() > 1e-3
    u = np.tile([0.3, -1.2, 0.5], (b.n, 1))
    u[:, dim:] = 0.0
    b.set(O.V, u)
    b.damp(40.0, 1e-5)
    assert np.abs(b.v - u).max() < 1e-13


def test_2d_layout_differs_from_paper_layout_and_threads_keep_bits():
    spec = S.BodySpec(dim=3, extent=(0.024, 0.008, 0.012), dp=1e-3, clamp_axis=0,
                      gravity=(0.0, -9.81, 0.0), beta=0.2, L_char=0.008, alpha=0.5, seed=4)
    a, _ = _body(spec, sweep_layout=O.SWEEP_2D)
    b, _ = _body(spec, sweep_layout=O.SWEEP_2D, threads=4)
    c, _ = _body(spec)
    for x in (a, b, c):
        x.step(10)
    assert a.damped_steps == c.damped_steps > 0
    assert np.array_equal(a.v, b.v) and np.array_equal(a.u, b.u)
    assert not np.array_equal(a.v, c.v)  # another order of the local operators
    assert np.abs(a.v - c.v).max() < 1e-2 * np.abs(c.v).max()


def test_both_layouts_relax_to_the_same_state():
    spec = S.BodySpec(dim=2, extent=(0.06, 0.012, 0), dp=0.002, clamp_axis=0, clamp_layers=3,
                      material=S.NEO_HOOKEAN, gravity=(0, -9.81, 0), beta=0.5, L_char=0.012,
                      alpha=0.2, seed=0)
    us = []
    for layout in (O.SWEEP_3D, O.SWEEP_2D):
        b, _ = _body(spec, sweep_layout=layout)
        st, steps, _ = b.relax(1e-13, 400000)
        assert st == 0
        us.append(b.u)
    assert np.abs(us[1] - us[0]).max() <= 5e-4 * np.abs(us[0]).max()
