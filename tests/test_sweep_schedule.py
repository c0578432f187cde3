"""The cell-wise synchronisation rule of the damping sweep, checked on the CPU.

The sweep S_d (Sec. 3.1) applies the local operators in the canonical order
of the splitting cell-linked list (Sec. 3.4): colours 0..3^d-1 forward, then
backward, the last non-empty colour's two directions fused.  Without grid
barriers, a cell runs its phase ph once every non-empty cell within 2 cells on
every axis (the cells whose 3^d footprints overlap its own) has finished the
directions it runs before ph; finished directions are counted over all sweeps
(2 per sweep, the fused phase counting both) on top of 2 x the epoch.

This test simulates that rule with groups of work items taken in phase order
(as the kernel's groups take them) and any interleaving of the groups, and
checks that (a) no interleaving deadlocks and (b) every pair of cells with
overlapping footprints runs in the canonical order, over consecutive sweeps.
It models the rule, not the kernel; the GPU tests check that the kernel gives
the barrier sweep's bits."""
import itertools
import random

import pytest


def colour(c, dim):
    x, y, z = c
    return x % 3 + 3 * (y % 3) + (9 * (z % 3) if dim == 3 else 0)


def phases_before(cy, ph, nc, clast):
    if cy == clast:
        return 2 if cy < ph else 0
    return (1 if cy < ph else 0) + (1 if 2 * nc - 1 - cy < ph else 0)


def neighbourhood(c, shape, dim):
    rng = range(-2, 3)
    for d in itertools.product(rng, rng, rng if dim == 3 else [0]):
        if d == (0, 0, 0):
            continue
        q = tuple(c[a] + d[a] for a in range(3))
        if all(0 <= q[a] < shape[a] for a in range(3)):
            yield q


def overlapping(a, b):
    return a != b and all(abs(a[k] - b[k]) <= 2 for k in range(3))


def simulate(shape, dim, occupied, ngroups, sweeps, seed, fused=None):
    """Run `sweeps` sweeps under the cell-wise rule with a random interleaving
    of the groups; return the global execution order of (sweep, phase, cell)
    or raise on a deadlock.  fused[s] is the colour whose two directions sweep
    s fuses: the body's own last colour alone, the batch's last colour (which
    may have no cell in this body) in a batch; default: the body's own."""
    rnd = random.Random(seed)
    nc = 27 if dim == 3 else 9
    cells_by_colour = [[] for _ in range(nc)]
    for c in sorted(occupied):
        cells_by_colour[colour(c, dim)].append(c)
    for lst in cells_by_colour:
        rnd.shuffle(lst)  # the kernel's colour lists have no set order
    own_last = max(k for k in range(nc) if cells_by_colour[k])
    done = {c: 0 for c in occupied}
    epoch = 0
    order = []
    for s in range(sweeps):
        clast = fused[s] if fused else own_last
        phases = []
        for ph in range(2 * nc):
            col = ph if ph < nc else 2 * nc - 1 - ph
            if not cells_by_colour[col] or (ph >= nc and col == clast):
                continue
            phases.append((ph, col))
        # group q takes items q, q + ngroups, ... of each phase, in phase order
        queues = [[] for _ in range(ngroups)]
        for ph, col in phases:
            for k, c in enumerate(cells_by_colour[col]):
                queues[k % ngroups].append((ph, col, c))
        heads = [0] * ngroups
        finished = 0
        total = sum(len(q) for q in queues)
        while finished < total:
            ready = []
            for g in range(ngroups):
                if heads[g] == len(queues[g]):
                    continue
                ph, col, c = queues[g][heads[g]]
                ok = all(done[q] >= 2 * epoch + phases_before(colour(q, dim), ph, nc, clast)
                         for q in neighbourhood(c, shape, dim) if q in occupied)
                if ok:
                    ready.append(g)
            if not ready:
                raise AssertionError(f"deadlock in sweep {s} after {finished} of {total} items")
            g = rnd.choice(ready)
            ph, col, c = queues[g][heads[g]]
            heads[g] += 1
            done[c] += 2 if col == clast else 1
            order.append((s, ph, c))
            finished += 1
        epoch += 1  # the last finisher advances the epoch
        assert all(v == 2 * epoch for v in done.values())
    return order


@pytest.mark.parametrize("dim,shape,fill,ngroups,seed", [
    (2, (7, 6, 1), 1.0, 3, 0), (2, (9, 5, 1), 0.6, 5, 1), (3, (5, 4, 4), 1.0, 4, 2),
    (3, (6, 5, 3), 0.55, 7, 3), (3, (4, 4, 4), 0.3, 2, 4), (2, (3, 2, 1), 1.0, 1, 5)])
def test_cellwise_rule_keeps_the_canonical_order(dim, shape, fill, ngroups, seed):
    rnd = random.Random(100 + seed)
    cells = [c for c in itertools.product(range(shape[0]), range(shape[1]), range(shape[2]))]
    occupied = {c for c in cells if rnd.random() < fill} or {cells[0]}
    for trial in range(3):
        order = simulate(shape, dim, occupied, ngroups, sweeps=2, seed=seed * 10 + trial)
        pos = {item: k for k, item in enumerate(order)}
        # canonical position of (sweep, phase): overlapping cells never share a
        # colour, so for them the phase index orders the operators
        for (s, ph, a), ka in pos.items():
            for (t, qh, b), kb in pos.items():
                if overlapping(a, b) and (s, ph) < (t, qh):
                    assert ka < kb, ((s, ph, a), (t, qh, b))


def test_overlapping_cells_never_share_a_colour():
    for dim in (2, 3):
        for a in itertools.product(range(6), range(6), range(6) if dim == 3 else [0]):
            for b in neighbourhood(a, (6, 6, 6 if dim == 3 else 1), dim):
                assert colour(a, dim) != colour(b, dim)



@pytest.mark.parametrize("dim,shape,fill,seed", [(2, (8, 2, 1), 0.9, 7), (3, (5, 5, 2), 0.8, 8),
                                                 (3, (4, 2, 3), 1.0, 9)])
def test_counts_stay_consistent_between_single_and_batched_sweeps(dim, shape, fill, seed):
    """A body alternates between single-body sweeps (its own last colour
    fused) and batched sweeps (the batch's last colour fused, possibly a
    colour the body has no cell of, so the body's own last colour runs its two
    directions apart).  Counting two directions per sweep keeps every wait
    satisfiable and the canonical order of each sweep."""
    rnd = random.Random(200 + seed)
    cells = [c for c in itertools.product(range(shape[0]), range(shape[1]), range(shape[2]))]
    occupied = {c for c in cells if rnd.random() < fill} or {cells[0]}
    nc = 27 if dim == 3 else 9
    own = max(colour(c, dim) for c in occupied)
    assert own < nc - 1  # the batch fuses a colour this body has no cell of
    fused = [own, nc - 1, own, nc - 1, nc - 1, own]
    order = simulate(shape, dim, occupied, 3, sweeps=len(fused), seed=seed, fused=fused)
    pos = {item: k for k, item in enumerate(order)}
    for (s, ph, a), ka in pos.items():
        for (t, qh, b), kb in pos.items():
            if overlapping(a, b) and (s, ph) < (t, qh):
                assert ka < kb, ((s, ph, a), (t, qh, b))
