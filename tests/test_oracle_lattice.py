"""Pins of the FP64 oracle's lattice-Boltzmann part (paper Sec. 2.1, 2.4).

Each test checks the oracle against something fixed by mathematics rather than
by the oracle itself: exact rational moment identities of the velocity set,
moment identities of the equilibrium and of the forcing term, conservation
laws, and closed-form steady flows (plane Poiseuille with its exact discrete
slip, Couette, rectangular-duct Fourier series).
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle


def test_velocity_set_isotropy():
    """D3Q19 (Sec. 2.1): weights and velocities give isotropic moments up to 4th order."""
    e, w, opp = oracle.constants()
    wf = [Fraction(x).limit_denominator(100) for x in w]
    assert sum(wf) == 1
    for a in range(3):
        assert sum(wf[i] * e[i, a] for i in range(19)) == 0
        for b in range(3):
            s2 = sum(wf[i] * e[i, a] * e[i, b] for i in range(19))
            assert s2 == (Fraction(1, 3) if a == b else 0)
            for c in range(3):
                assert sum(wf[i] * e[i, a] * e[i, b] * e[i, c] for i in range(19)) == 0
                for d in range(3):
                    s4 = sum(wf[i] * e[i, a] * e[i, b] * e[i, c] * e[i, d] for i in range(19))
                    expect = Fraction(int(a == b and c == d) + int(a == c and b == d) + int(a == d and b == c), 9)
                    assert s4 == expect
    for i in range(19):
        assert np.array_equal(e[opp[i]], -e[i])
    assert len({tuple(v) for v in e}) == 19


def test_equilibrium_moments():
    """f^eq reproduces rho, rho u and rho (I/3 + u u)."""
    rng = np.random.default_rng(3)
    e, w, _ = oracle.constants()
    for _ in range(20):
        rho = 0.8 + 0.4 * rng.random()
        u = 0.1 * rng.standard_normal(3)
        feq = oracle.equilibrium(rho, u)
        assert abs(feq.sum() - rho) < 1e-15
        np.testing.assert_allclose(feq @ e, rho * u, atol=1e-15)
        P = np.einsum("i,ia,ib->ab", feq, e, e)
        np.testing.assert_allclose(P, rho * (np.eye(3) / 3 + np.outer(u, u)), atol=1e-15)


def test_guo_source_moments():
    """Guo forcing: zeroth moment 0, first (1 - 1/2tau) g, second (1 - 1/2tau)(u g + g u)."""
    rng = np.random.default_rng(4)
    e, _, _ = oracle.constants()
    for tau in (0.6, 1.0, 1.7):
        for _ in range(10):
            u = 0.05 * rng.standard_normal(3)
            g = 1e-3 * rng.standard_normal(3)
            S = oracle.guo_source(tau, u, g)
            pre = 1 - 1 / (2 * tau)
            assert abs(S.sum()) < 1e-18
            np.testing.assert_allclose(S @ e, pre * g, atol=1e-18)
            np.testing.assert_allclose(np.einsum("i,ia,ib->ab", S, e, e),
                                       pre * (np.outer(u, g) + np.outer(g, u)), atol=1e-18)


def _spheres():
    return np.array([[5.0, 6.0, 4.0, 2.5], [11.5, 4.25, 6.0, 2.0]], np.float32)


def test_rasterise_bruteforce():
    """Obstacle nodes (Sec. 2.4/2.5) = lattice points inside or on a sphere."""
    dims = (16, 12, 10)
    sph = _spheres()
    solid = oracle.rasterise(sph, dims).reshape(dims[2], dims[1], dims[0])
    for z in range(dims[2]):
        for y in range(dims[1]):
            for x in range(dims[0]):
                inside = any((x - s[0]) ** 2 + (y - s[1]) ** 2 + (z - s[2]) ** 2 <= s[3] ** 2 for s in sph.astype(float))
                assert solid[z, y, x] == inside
    # a point exactly on the surface counts as solid
    on = oracle.rasterise(np.array([[2.0, 2.0, 2.0, 2.0]], np.float32), (6, 6, 6)).reshape(6, 6, 6)
    assert on[2, 2, 4] == 1 and on[2, 2, 5] == 0


def test_rest_state_stays_at_equilibrium():
    """rho = 1, u = 0, no force: walls and obstacles leave f^eq unchanged (1e-14), 1000 steps."""
    dims = (16, 12, 10)
    s = oracle.System(dims, tau=1.0, periodic=(1, 0, 0))
    s.set_solid(oracle.rasterise(_spheres(), dims))
    s.step(1000)
    f = s.get_f()
    _, w, _ = oracle.constants()
    fluid = s.solid == 0
    assert np.abs(f[:, fluid] - w[:, None]).max() < 1e-14


def _random_state(s, seed, amp=1e-3):
    rng = np.random.default_rng(seed)
    f = s.get_f()
    f = f * (1 + amp * rng.standard_normal(f.shape))
    s.set_f(f)


def test_mass_conservation_with_walls_obstacles_and_force():
    dims = (16, 12, 10)
    s = oracle.System(dims, tau=0.9, body_force=(1e-4, 2e-5, 0.0), periodic=(1, 0, 0))
    s.set_solid(oracle.rasterise(_spheres(), dims))
    _random_state(s, 1)
    g = np.random.default_rng(2).standard_normal((3, s.N)) * 1e-4
    g[:, s.solid == 1] = 0
    s.set_extra_force(g)
    fluid = s.solid == 0
    m0 = s.get_f()[:, fluid].sum()
    s.step(200)
    m1 = s.get_f()[:, fluid].sum()
    assert abs(m1 - m0) / m0 < 1e-13


def test_momentum_budget_periodic_box():
    """Fully periodic: P(t+1) - P(t) = sum_x g(x) exactly (Guo forcing + half-force velocity)."""
    dims = (8, 6, 5)
    e, _, _ = oracle.constants()
    s = oracle.System(dims, tau=0.8, periodic=(1, 1, 1))
    _random_state(s, 5)
    g = np.random.default_rng(6).standard_normal((3, s.N)) * 1e-4
    s.set_extra_force(g)
    P0 = np.einsum("ip,id->d", s.get_f(), e)
    for k in range(1, 6):
        s.step(1)
        P = np.einsum("ip,id->d", s.get_f(), e)
        np.testing.assert_allclose(P - P0, k * g.sum(axis=1), rtol=0, atol=2e-13)


@pytest.mark.parametrize("H", [8, 16])
@pytest.mark.parametrize("tau", [0.8, 1.0, 1.5, 0.5 + (3 / 16) ** 0.5])
def test_plane_poiseuille_exact_discrete_solution(H, tau):
    """Walls at y = -1/2 and y = H - 1/2 (halfway bounce-back, Sec. 2.4), force G in x.

    The steady BGK + Guo solution is exactly
    u(y) = G/(2 nu) (y + 1/2)(H - 1/2 - y) + G (16 L - 3)/(24 nu),
    nu = (tau - 1/2)/3, L = (tau - 1/2)^2: a parabola plus a tau-dependent slip.
    """
    G = 1e-4
    s = oracle.System((1, H, 1), tau=tau, body_force=(G, 0, 0), periodic=(1, 0, 1))
    nu = (tau - 0.5) / 3
    L = (tau - 0.5) ** 2
    y = np.arange(H)
    exact = G / (2 * nu) * (y + 0.5) * (H - 0.5 - y) + G * (16 * L - 3) / (24 * nu)
    prev = None
    for _ in range(400):
        s.step(200)
        _, u = s.fields()
        if prev is not None and np.abs(u[0] - prev).max() < 1e-15 * exact.max():
            break
        prev = u[0].copy()
    assert np.abs(u[0] - exact).max() / exact.max() < 2e-12
    assert np.abs(u[1:]).max() < 1e-12 * exact.max()


def test_plane_poiseuille_second_order_at_tau_one():
    """At tau = 1 the slip is G/4: relative error vs the continuum parabola falls 4x per doubling."""
    errs = []
    for H in (8, 16, 32):
        G = 1e-5
        s = oracle.System((1, H, 1), tau=1.0, body_force=(G, 0, 0), periodic=(1, 0, 1))
        s.step(int(40 * H * H))
        _, u = s.fields()
        y = np.arange(H)
        cont = G * 3 * (y + 0.5) * (H - 0.5 - y)
        errs.append(np.linalg.norm(u[0] - cont) / np.linalg.norm(cont))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.7 < r1 < 4.3 and 3.7 < r2 < 4.3


@pytest.mark.parametrize("tau", [0.8, 1.0, 1.5])
def test_couette_linear_profile(tau):
    """Moving upper wall (Ladd term): u_x = U (y + 1/2)/H at steady state, exactly."""
    H, U = 16, 1e-3
    s = oracle.System((1, H, 1), tau=tau, periodic=(1, 0, 1), wall_velocity=((0, 0, 0), (U, 0, 0)))
    s.step(20000)
    rho, u = s.fields()
    y = np.arange(H)
    assert np.abs(u[0] - U * (y + 0.5) / H).max() / U < 1e-10
    assert np.abs(rho - 1).max() < 1e-11


def _duct_series(ny, nz, G, nu, nterm=200):
    a, b = ny / 2, nz / 2
    y = np.arange(ny) - (ny - 1) / 2
    z = np.arange(nz) - (nz - 1) / 2
    Y, Z = np.meshgrid(y, z, indexing="xy")
    u = np.zeros_like(Y)
    for n in range(1, 2 * nterm, 2):
        k = n * np.pi / (2 * a)
        u += (-1) ** ((n - 1) // 2) / n ** 3 * (1 - np.cosh(k * Z) / np.cosh(k * b)) * np.cos(k * Y)
    return 16 * G * a * a / (nu * np.pi ** 3) * u


def test_rectangular_duct_second_order():
    """Walls in y and z (the plain channel's cross-section): steady flow vs the Fourier series."""
    errs = []
    for ny in (8, 16, 32):
        G, tau = 1e-6, 1.0
        nu = (tau - 0.5) / 3
        s = oracle.System((1, ny, ny), tau=tau, body_force=(G, 0, 0), periodic=(1, 0, 0))
        s.step(int(30 * ny * ny / (nu * np.pi ** 2 * 2)))
        _, u = s.fields()
        ex = _duct_series(ny, ny, G, nu)
        errs.append(np.linalg.norm(u[0].reshape(ny, ny) - ex) / np.linalg.norm(ex))
    assert errs[0] < 1e-2
    assert 3.0 < errs[0] / errs[1] < 4.5 and 3.4 < errs[1] / errs[2] < 4.5
