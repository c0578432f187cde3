"""Pins of the oracle's closed pieces against mathematics the paper fixes.

Kernel (Sec. 4 intro: 5th-order Wendland C2, h = 1.3 dp), material constants
(Eq. modulus-relation), constitutive laws (Eqs. constitutive-equation,
strain-density, PK-stress), viscosity parameter (Eq. viscous-parameter), the
Philox4x64-10 random stream (random choice, Sec. 3.3) and the time-step
criterion (Eq. time-step-criterion, Eq. viscous-criteria).
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, linalg

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ kernel
@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("h", [1.0, 1.3e-3])
def test_kernel_normalised(dim, h):
    # a smoothing kernel integrates to one over its support
    if dim == 2:
        val, _ = integrate.quad(lambda r: 2 * math.pi * r * O.kernel_W(2, h, r), 0, 2 * h,
                                epsabs=0, epsrel=1e-13)
    else:
        val, _ = integrate.quad(lambda r: 4 * math.pi * r * r * O.kernel_W(3, h, r), 0, 2 * h,
                                epsabs=0, epsrel=1e-13)
    assert abs(val - 1.0) < 1e-10


@pytest.mark.parametrize("dim", [2, 3])
def test_kernel_derivative_matches_finite_difference(dim):
    h = 1.3
    for r in np.linspace(0.05, 2 * h - 0.05, 23):
        e = 1e-6
        fd = (O.kernel_W(dim, h, r + e) - O.kernel_W(dim, h, r - e)) / (2 * e)
        assert abs(O.kernel_dW(dim, h, r) - fd) <= 1e-7 * max(1.0, abs(fd))


@pytest.mark.parametrize("dim", [2, 3])
def test_kernel_support_and_sign(dim):
    h = 0.7
    assert O.kernel_W(dim, h, 2 * h) == 0.0
    assert O.kernel_dW(dim, h, 2 * h) == 0.0
    assert O.kernel_W(dim, h, 2.5 * h) == 0.0
    assert O.kernel_dW(dim, h, 0.0) == 0.0
    for r in np.linspace(1e-3, 2 * h - 1e-3, 50):
        assert O.kernel_W(dim, h, r) > 0.0
        assert O.kernel_dW(dim, h, r) < 0.0


def test_kernel_c2_at_support_edge():
    # C2 smoothness: W, W' and W'' vanish at q = 2
    h = 1.0
    e = 1e-4
    w2 = (O.kernel_dW(3, h, 2 - e) - O.kernel_dW(3, h, 2 - 2 * e)) / e
    assert abs(O.kernel_W(3, h, 2 - e)) < 1e-12
    assert abs(O.kernel_dW(3, h, 2 - e)) < 1e-9
    assert abs(w2) < 1e-4


# ------------------------------------------------------------------ material constants
@pytest.mark.parametrize("E,nu", [(2e6, 0.3), (1e6, 0.45), (5e4, 0.45), (6.75e10, 0.34)])
def test_lame_constants_textbook(E, nu):
    lam, mu = O.lame(E, nu)
    # textbook definitions of Young's modulus and Poisson's ratio
    assert abs(mu * (3 * lam + 2 * mu) / (lam + mu) - E) <= 1e-12 * E
    assert abs(lam / (2 * (lam + mu)) - nu) <= 1e-14
    # second equality of Eq. modulus-relation (printed correctly): E = 3K(1 - 2 nu)
    K = lam + 2 * mu / 3
    assert abs(3 * K * (1 - 2 * nu) - E) <= 1e-12 * E


def test_lame_known_values():
    lam, mu = O.lame(2e6, 0.3)
    assert abs(mu - 2e6 / 2.6) < 1e-6
    assert abs(lam - 2e6 * 0.3 / (1.3 * 0.4)) < 1e-6


# ------------------------------------------------------------------ constitutive laws
def _rot3(a, b, c):
    return linalg.expm(np.array([[0, -c, b], [c, 0, -a], [-b, a, 0]], dtype=float))


@pytest.mark.parametrize("material", [O.SVK, O.NEO_HOOKEAN])
@pytest.mark.parametrize("dim", [2, 3])
def test_rigid_rotation_is_stress_free(material, dim):
    lam, mu = O.lame(2e6, 0.3)
    if dim == 3:
        R = _rot3(0.3, -1.1, 0.7)
    else:
        t = 0.9
        R = np.array([[math.cos(t), -math.sin(t), 0], [math.sin(t), math.cos(t), 0], [0, 0, 1.0]])
    S = O.pk2(dim, material, lam, mu, R)
    assert np.abs(S).max() < 1e-9 * mu


def _energy_svk(dim, lam, mu, Emat):
    # Saint-Venant-Kirchhoff energy, textbook: lambda/2 (tr E)^2 + mu E:E
    E = Emat[:dim, :dim]
    return 0.5 * lam * np.trace(E) ** 2 + mu * np.sum(E * E)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("material", [O.SVK, O.NEO_HOOKEAN])
def test_pk2_is_energy_derivative(dim, material):
    """S = dW/dE by central differences in E (Eq. PK-stress); the neo-Hookean
    energy is the oracle's transcription of Eq. strain-density, the SVK energy
    the textbook one.  F is recovered from C = I + 2E by a symmetric square
    root (any F with F^T F = C gives the same S)."""
    lam, mu = O.lame(1e6, 0.45)
    rng = np.random.default_rng(5)
    A = rng.normal(scale=0.08, size=(dim, dim))
    E0 = 0.5 * (A + A.T)

    def W(E):
        C = np.eye(dim) + 2 * E
        F = np.real(linalg.sqrtm(C))
        if material == O.SVK:
            return _energy_svk(dim, lam, mu, E)
        return O.nh_energy(dim, lam, mu, F)

    F0 = np.real(linalg.sqrtm(np.eye(dim) + 2 * E0))
    S = O.pk2(dim, material, lam, mu, F0)
    e = 1e-6
    for a in range(dim):
        for b in range(dim):
            dE = np.zeros((dim, dim))
            dE[a, b] += 0.5 * e
            dE[b, a] += 0.5 * e
            dW = (W(E0 + dE) - W(E0 - dE)) / (2 * e)
            # dW = S : dE / e = S_ab (S symmetric)
            assert abs(dW - S[a, b]) <= 2e-5 * mu, (a, b, dW, S[a, b])


@pytest.mark.parametrize("dim", [2, 3])
def test_neo_hookean_and_svk_agree_at_small_strain(dim):
    lam, mu = O.lame(2e6, 0.3)
    rng = np.random.default_rng(11)
    G = rng.normal(size=(dim, dim))
    prev = None
    for eps in [1e-2, 1e-3, 1e-4]:
        F = np.eye(3)
        F[:dim, :dim] += eps * G
        s1 = O.pk2(dim, O.SVK, lam, mu, F)
        s2 = O.pk2(dim, O.NEO_HOOKEAN, lam, mu, F)
        rel = np.abs(s1 - s2).max() / np.abs(s1).max()
        assert rel < 10 * eps
        if prev is not None:
            assert rel < 0.2 * prev  # difference is O(eps^2) against O(eps) stress
        prev = rel


def test_cauchy_stress_symmetric():
    # P = F S with S symmetric makes sigma = P F^T / J symmetric (Eq. piola)
    lam, mu = O.lame(2e6, 0.3)
    rng = np.random.default_rng(2)
    for material in [O.SVK, O.NEO_HOOKEAN]:
        F = np.eye(3) + rng.normal(scale=0.1, size=(3, 3))
        S = O.pk2(3, material, lam, mu, F)
        assert np.abs(S - S.T).max() < 1e-9 * mu
        sig = F @ S @ F.T
        assert np.abs(sig - sig.T).max() < 1e-9 * mu


# ------------------------------------------------------------------ viscosity parameter
def test_viscosity_parameter_golden():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "viscosity_parameter.txt"))
            if l.strip() and not l.startswith("#")]
    for beta, rho, E, L, printed, digits in rows:
        val = O.eta(float(beta), float(rho), float(E), float(L))
        assert float(f"{val:.{int(digits)}g}") == float(printed)


# ------------------------------------------------------------------ Philox4x64-10
def test_philox_matches_numpy_bit_generator():
    """numpy.random.Philox is Philox4x64-10; it increments its 256-bit counter
    before producing a block, so our block at counter c equals numpy's first
    block after constructing it with counter c - 1."""
    for seed in [0, 1, 2, 3, 12345, 2**63 + 17, 2**64 - 1]:
        for step in [1, 2, 3, 1000, 2**40 + 3]:
            mine = O.philox4x64_10([step, 0, 0, 0], [seed, 0])
            bg = np.random.Philox(key=np.array([seed, 0], dtype=np.uint64),
                                  counter=np.array([step - 1, 0, 0, 0], dtype=np.uint64))
            assert list(mine) == list(bg.random_raw(4))
    # counter 0 = numpy's all-ones counter incremented (carry through all words)
    mine = O.philox4x64_10([0, 0, 0, 0], [7, 0])
    ones = np.array([2**64 - 1] * 4, dtype=np.uint64)
    bg = np.random.Philox(key=np.array([7, 0], dtype=np.uint64), counter=ones)
    assert list(mine) == list(bg.random_raw(4))


def test_random_choice_fraction():
    # phi uniform in [0, 1): damped fraction within alpha +- 4 sigma
    n = 200000
    for seed in [0, 1]:
        phis = np.array([O.phi(seed, s) for s in range(n)])
        assert phis.min() >= 0.0 and phis.max() < 1.0
        for alpha in [0.2, 0.5]:
            frac = np.mean(phis < alpha)
            sig = math.sqrt(alpha * (1 - alpha) / n)
            assert abs(frac - alpha) < 4 * sig


# ------------------------------------------------------------------ time step
def test_time_step_criterion_closed_form():
    """Eq. time-step-criterion with |v|max = 0, |a|max = g, and the implicit
    viscous limit of Eq. viscous-criteria; 2D cantilever numbers."""
    dp = 0.002
    h = 1.3 * dp
    E, nu, rho, g = 2e6, 0.3, 1000.0, 9.81
    r0 = np.array([[(i + 0.5) * dp, (j + 0.5) * dp] for j in range(6) for i in range(6)])
    p = O.Params(dim=2, material=O.SVK, rho0=rho, E=E, nu=nu, h=h, gravity=(0, -g, 0),
                 beta=0.2, L_char=0.02, alpha=0.2)
    b = O.OracleBody(p, r0, vol_default=dp * dp)
    K = E / (3 * (1 - 2 * nu))
    c = math.sqrt(K / rho)
    acoustic = 0.6 * min(h / c, math.sqrt(h / g))
    eta = 0.25 * 0.2 * math.sqrt(rho * E) * 0.02
    viscous = 50 * h * h / (eta / (0.2 * rho) * 2)
    assert abs(b.dt - min(acoustic, viscous)) <= 1e-15
    assert abs(b.dt - 3.8212e-5) < 1e-9
    # a viscosity large enough to bind the viscous limit
    p.beta = 20.0
    b2 = O.OracleBody(p, r0, vol_default=dp * dp)
    eta2 = 0.25 * 20.0 * math.sqrt(rho * E) * 0.02
    assert abs(b2.dt - 50 * h * h / (eta2 / (0.2 * rho) * 2)) <= 1e-15
