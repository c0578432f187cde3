"""The oracle's OpenMP build against its serial build: the per-particle
loops and the cells of one sweep colour run on several threads, which must
change no bit (each particle's sums keep their order; the cells of a colour
touch disjoint particles, Sec. 3.4; the kinetic energy is summed serially)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2103_08932_gb300 import synth as S


def _body(spec, threads, damping=O.DAMP_PARTICLE, jitter=0.0):
    r0, flags, _ = S.jittered(spec, jitter, 9) if jitter > 0 else S.lattice(spec)
    p = O.Params(dim=spec.dim, material=spec.material, rho0=spec.rho0, E=spec.E, nu=spec.nu,
                 h=spec.h, gravity=spec.gravity, beta=spec.beta, L_char=spec.L_char,
                 alpha=spec.alpha, seed=spec.seed, damping=damping)
    return O.OracleBody(p, r0[:, :spec.dim], vol_default=spec.vol, flags=flags, threads=threads)


@pytest.mark.parametrize("dim,damping,jitter", [(3, O.DAMP_PARTICLE, 0.0), (3, O.DAMP_PAIRWISE, 0.3),
                                                (2, O.DAMP_PARTICLE, 0.2)])
def test_openmp_build_is_bitwise_serial(dim, damping, jitter):
    if dim == 3:
        spec = S.BodySpec(dim=3, extent=(0.024, 0.008, 0.012), dp=1e-3, clamp_axis=0,
                          gravity=(0.0, -9.81, 0.0), beta=0.2, L_char=0.008, alpha=0.5, seed=4)
    else:
        spec = S.BodySpec(dim=2, extent=(0.06, 0.01, 0.0), dp=1e-3, clamp_axis=0, material=S.SVK,
                          gravity=(0.0, -9.81, 0.0), beta=0.2, L_char=0.01, alpha=0.5, seed=4)
    a = _body(spec, 0, damping, jitter)
    b = _body(spec, 4, damping, jitter)
    a.step(12)
    b.step(12)
    assert a.damped_steps == b.damped_steps > 0
    assert np.array_equal(a.v, b.v)
    assert np.array_equal(a.u, b.u)
    assert a.ke == b.ke
