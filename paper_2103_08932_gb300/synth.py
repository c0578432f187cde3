"""Seeded synthetic inputs: lattice bodies and the benchmark workloads.

This module holds none of the method's arithmetic.  It only lays particles on
a lattice (centres at (i + 1/2) dp), marks constrained and end-loaded
particles, writes the initial displacement of a prescribed-displacement body,
and lists the parameter sets of the workloads.  Both the CUDA library's tests
and the oracle's tests draw their inputs from here; it imports nothing from
either.

Particle order ("original order"): z outermost, then y, then x innermost, the
constrained layers included in the index ranges.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

FLAG_CONSTRAINED = 1
FLAG_END_LOAD = 2

SVK = 0
NEO_HOOKEAN = 1


@dataclass
class BodySpec:
    """A box-shaped body on a cubic lattice of spacing dp.

    The body occupies [0, extent[a]) along each axis.  ``clamp_layers`` extra
    lattice layers lie below 0 on ``clamp_axis`` and are held fixed
    (u = 0, v = 0).  ``presc_layers`` extra layers lie beyond extent on the
    same axis and are held at displacement ``presc_disp``; the body particles
    then start from the linear interpolation between the two constrained faces.
    ``end_load`` particles are the body's last lattice layer on ``clamp_axis``.
    """
    dim: int = 3
    extent: tuple = (0.2, 0.02, 0.1)
    dp: float = 1e-3
    clamp_axis: int = 0
    clamp_layers: int = 3
    presc_layers: int = 0
    presc_disp: tuple = (0.0, 0.0, 0.0)
    end_load_layer: bool = False
    # material and load
    material: int = NEO_HOOKEAN
    rho0: float = 1000.0
    E: float = 2e6
    nu: float = 0.3
    h_over_dp: float = 1.3
    gravity: tuple = (0.0, -9.81, 0.0)
    end_load: tuple = (0.0, 0.0, 0.0)
    # relaxation
    beta: float = 0.2
    L_char: float = 0.02
    alpha: float = 0.2
    seed: int = 0
    # rotational body force (gamma0, L, y_c, z_c) of the twisting cantilever
    twist: tuple = (0.0, 0.0, 0.0, 0.0)

    def counts(self):
        n = [1, 1, 1]
        for a in range(self.dim):
            n[a] = int(round(self.extent[a] / self.dp))
        return n

    @property
    def h(self) -> float:
        return self.h_over_dp * self.dp

    @property
    def vol(self) -> float:
        return self.dp ** self.dim


def lattice(spec: BodySpec):
    """Return (r0 (n,3) float64, flags (n,) uint8, u0 (n,3) float64)."""
    dim = spec.dim
    n = spec.counts()
    lo = [0, 0, 0]
    hi = [n[0], n[1], n[2]]
    ax = spec.clamp_axis
    if ax >= 0:
        lo[ax] = -spec.clamp_layers
        hi[ax] = n[ax] + spec.presc_layers
    idx = [np.arange(lo[a], hi[a]) for a in range(3)]
    if dim == 2:
        idx[2] = np.arange(0, 1)
    gz, gy, gx = np.meshgrid(idx[2], idx[1], idx[0], indexing="ij")
    ijk = np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1)
    r0 = (ijk.astype(np.float64) + 0.5) * spec.dp
    if dim == 2:
        r0[:, 2] = 0.0
    flags = np.zeros(len(r0), dtype=np.uint8)
    u0 = np.zeros((len(r0), 3))
    if ax >= 0:
        k = ijk[:, ax]
        flags[k < 0] |= FLAG_CONSTRAINED
        flags[k >= n[ax]] |= FLAG_CONSTRAINED
        if spec.end_load_layer:
            flags[k == n[ax] - 1] |= FLAG_END_LOAD
        if spec.presc_layers > 0:
            d = np.asarray(spec.presc_disp, dtype=np.float64)
            length = n[ax] * spec.dp
            frac = np.clip(r0[:, ax] / length, 0.0, 1.0)
            frac[k < 0] = 0.0
            frac[k >= n[ax]] = 1.0
            u0 = frac[:, None] * d[None, :]
            if dim == 2:
                u0[:, 2] = 0.0
    return r0, flags, u0


def jittered(spec: BodySpec, amplitude: float, seed: int):
    """Lattice positions moved by a seeded uniform jitter of +-amplitude*dp."""
    r0, flags, u0 = lattice(spec)
    rng = np.random.default_rng(seed)
    j = rng.uniform(-amplitude, amplitude, size=r0.shape) * spec.dp
    if spec.dim == 2:
        j[:, 2] = 0.0
    return r0 + j, flags, u0


# ------------------------------------------------------------------ workloads
def cantilever_2d(material: int = NEO_HOOKEAN) -> BodySpec:
    """2D cantilever under gravity: L = 0.2 m, H = 0.02 m, dp = H/10,
    100 x 10 body particles + 3 clamped columns, E = 2e6 Pa, nu = 0.3,
    rho = 1000 kg/m^3, g = 9.81 m/s^2, beta = alpha = 0.2, seed 0."""
    return BodySpec(dim=2, extent=(0.2, 0.02, 0.0), dp=0.002, clamp_axis=0, clamp_layers=3,
                    material=material, rho0=1000.0, E=2e6, nu=0.3, gravity=(0.0, -9.81, 0.0),
                    beta=0.2, L_char=0.02, alpha=0.2, seed=0)


def cantilever_plate_3d(dp: float = 1e-3) -> BodySpec:
    """3D cantilever plate 0.2 x 0.02 x 0.1 m, dp = 1 mm (200 x 20 x 100 body
    particles + 3 clamped layers at x < 0, 406,000 in all), gravity along -y,
    same material as the 2D cantilever, alpha = 0.2, seed 1."""
    return BodySpec(dim=3, extent=(0.2, 0.02, 0.1), dp=dp, clamp_axis=0, clamp_layers=3,
                    material=NEO_HOOKEAN, rho0=1000.0, E=2e6, nu=0.3, gravity=(0.0, -9.81, 0.0),
                    beta=0.2, L_char=0.02, alpha=0.2, seed=1)


def twisting_cantilever_3d(dp: float = 1e-3) -> BodySpec:
    """Twisting cantilever: a 0.2 m beam of square 0.02 m section, dp = 1 mm
    (200 x 20 x 20 body particles + 3 clamped layers, 81,200 in all),
    neo-Hookean as the bending case, no gravity, the rotational body force
    about the beam axis with gamma0 = 20 g / H (g = 9.8, H = 0.02 m), seed 5."""
    H = 0.02
    return BodySpec(dim=3, extent=(0.2, H, H), dp=dp, clamp_axis=0, clamp_layers=3,
                    material=NEO_HOOKEAN, rho0=1000.0, E=2e6, nu=0.3, gravity=(0.0, 0.0, 0.0),
                    beta=0.2, L_char=H, alpha=0.2, seed=5, twist=(20 * 9.8 / H, 0.2, H / 2, H / 2))


def compression_block_3d(dp: float = 8e-4, edge: float = 0.1) -> BodySpec:
    """3D block compression: cube of edge 0.1 m, dp = 0.8 mm (125^3 body
    particles), neo-Hookean E = 1e6 Pa, nu = 0.45, rho = 1000 kg/m^3, bottom
    face fixed (3 layers), top face displaced by -10 % of the height (3
    layers), no gravity, seed 2."""
    return BodySpec(dim=3, extent=(edge, edge, edge), dp=dp, clamp_axis=2, clamp_layers=3,
                    presc_layers=3, presc_disp=(0.0, 0.0, -0.1 * edge), material=NEO_HOOKEAN,
                    rho0=1000.0, E=1e6, nu=0.45, gravity=(0.0, 0.0, 0.0), beta=0.2, L_char=edge,
                    alpha=0.2, seed=2)


def scaled(spec: BodySpec, factor: float) -> BodySpec:
    """The same body with every length multiplied by ``factor`` at the same
    lattice spacing (fewer particles, same per-particle physics)."""
    ext = tuple(e * factor for e in spec.extent)
    return replace(spec, extent=ext, L_char=spec.L_char * factor)


def random_bodies(count: int, n_lo: float, n_hi: float, seed: int):
    """Uneven bodies: particle counts log-uniform in [n_lo, n_hi], each a box,
    beam or plate with aspect ratios in [1, 20], dp from the count, E
    log-uniform in [1e5, 1e7] Pa, nu uniform in [0.2, 0.45], loaded by gravity
    or by an end load."""
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        n_target = math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))
        shape = int(rng.integers(0, 3))  # 0 box, 1 beam, 2 plate
        asp = rng.uniform(1.0, 20.0)
        if shape == 0:
            rel = np.array([1.0, rng.uniform(1.0, 2.0), rng.uniform(1.0, 2.0)])
        elif shape == 1:
            rel = np.array([asp, 1.0, 1.0])
        else:
            rel = np.array([asp, 1.0, asp * rng.uniform(0.3, 1.0)])
        # at least 6 layers thick (the kernel support spans 5.2 dp: thinner
        # bodies are under-resolved and the method diverges on them, oracle
        # included); counts from the target particle number
        scale = (n_target / np.prod(rel)) ** (1.0 / 3.0)
        cnt = np.maximum(np.round(rel * scale).astype(int), 6)
        length = 0.1
        dp = length / cnt[0]
        E = math.exp(rng.uniform(math.log(1e5), math.log(1e7)))
        nu = rng.uniform(0.2, 0.45)
        load = int(rng.integers(0, 2))
        thickness = float(cnt.min()) * dp
        # loads capped so that the linear cantilever tip deflection stays
        # below 5 % of the length (slender soft beams would otherwise fold)
        rho0, span, hy = 1000.0, float(cnt[0]) * dp, float(cnt[1]) * dp
        g_cap = 0.05 * 2.0 * E * hy * hy / (3.0 * rho0 * span ** 3)
        a_cap = 0.05 * E * hy * hy / (4.0 * rho0 * dp * span * span)
        g = min(9.81, g_cap)
        a_end = min(50.0, a_cap)
        spec = BodySpec(dim=3, extent=tuple(float(c) * dp for c in cnt), dp=dp, clamp_axis=0,
                        clamp_layers=3, material=NEO_HOOKEAN, rho0=rho0, E=E, nu=nu,
                        gravity=(0.0, -g, 0.0) if load == 0 else (0.0, 0.0, 0.0),
                        end_load=(0.0, 0.0, 0.0) if load == 0 else (0.0, -a_end, 0.0),
                        end_load_layer=(load == 1), beta=0.2, L_char=thickness, alpha=0.2,
                        seed=seed * 100003 + b)
        out.append(spec)
    return out


def poisson_arrivals(rate: float, count: int, seed: int):
    """Arrival times (s) of a Poisson request stream."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))
