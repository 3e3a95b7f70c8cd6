"""Pins of the oracle's IB points with mass (Sec. 2.2: m d^2X/dt^2 = F, the
coupling force from the motion of the point relative to the fluid; reading: a
kick by the membrane force, then a drift under the drag -gamma (V - U) solved
exactly with U held, the fluid receiving the drag's impulse).

* the drift coefficients p1 = (1 - e^-a)/a and e^-a against 40-digit
  evaluations (both branches of the oracle's formula);
* one step of a force-free cell in a uniformly moving periodic fluid: every
  node reaches V = u0 (1 - e^-a) and moves u0 (1 - (1 - e^-a)/a), the closed
  form of the drag ODE (U is exactly u0 by the partition of unity);
* total momentum (fluid populations + m * point velocities) is conserved to
  round-off in a periodic box with a deforming cell: the fluid gains exactly
  the impulse the points lose (a dropped p1, a wrong sign or a missing
  (1 - p1) breaks it);
* gamma = 0: nothing reaches the fluid (bit-identical to the same fluid
  without the cell), the cell's centroid does not move (internal forces sum
  to zero) and the leapfrog step keeps the deforming cell bounded;
* m -> 0: the impulse equals the membrane force, so the first cycle's fluid
  update is the massless cycle's, and the points move by F / gamma.
"""
import numpy as np
import pytest

import oracle
from paper_1110_0995_gb300 import scene


def _cell(scale=2.2, centre=(6.3, 6.1, 5.9), amp=0.0, seed=0):
    x, t = scene.icosphere(1)
    rng = np.random.default_rng(seed)
    x0 = scale * x + np.array(centre)
    xd = x0 + amp * rng.standard_normal(x0.shape)
    return x0, xd, t


MOD = (0.02, 0.01, 0.01, 0.5, 0.9)


@pytest.mark.parametrize("a", [1e-7, 1e-4, 9.99e-4, 1e-3, 0.02, 0.5, 1.0, 7.0, 40.0])
def test_drag_coefficients_against_40_digits(a):
    sympy = pytest.importorskip("sympy")
    A = sympy.Rational(repr(a))
    e = sympy.exp(-A)
    p1 = float(sympy.N((1 - e) / A, 40))
    E = float(sympy.N(e, 40))
    got = oracle.drag_coefficients(1.0, a)
    assert got[0] == a
    assert got[1] == pytest.approx(p1, rel=1e-14)
    assert got[2] == pytest.approx(E, rel=1e-15)


@pytest.mark.parametrize("m,gamma", [(1.0, 0.5), (0.3, 2.0), (5.0, 1e-5)])
def test_one_step_closed_form_in_uniform_flow(m, gamma):
    x0, _, t = _cell()
    u0 = np.array([0.012, -0.004, 0.007])
    s = oracle.System((14, 12, 12), 1.0, (0, 0, 0), (1, 1, 1))
    s.init_equilibrium(1.0, u0)
    s.add_mesh(x0, t, MOD)
    s.set_dynamics(m, gamma)
    s.step(1)
    a = gamma / m
    v_exact = u0 * (-np.expm1(-a))
    dx_exact = u0 * (1.0 + np.expm1(-a) / a)
    assert np.abs(s.velocities(0) - v_exact).max() < 1e-15
    assert np.abs(s.nodes(0) - x0 - dx_exact).max() < 2e-15


def test_total_momentum_conserved():
    x0, xd, t = _cell(amp=0.15, seed=3)
    m, gamma = 0.7, 0.4
    s = oracle.System((14, 12, 12), 0.9, (0, 0, 0), (1, 1, 1))
    s.add_mesh(x0, t, MOD)
    s.set_nodes(0, xd)
    s.set_dynamics(m, gamma)
    e, _, _ = oracle.constants()

    def momentum():
        f = s.get_f()
        return (e.T.astype(float) @ f).sum(axis=1) + m * s.velocities(0).sum(axis=0)

    p0 = momentum()
    moved = 0.0
    for _ in range(25):
        s.step(1)
        moved = max(moved, np.abs(m * s.velocities(0)).sum())
        # round-off of the lattice sums (38,000 populations), against an exchange of ~1e-3 per step
        assert np.abs(momentum() - p0).max() < 1e-11
    assert moved > 1e-4      # the points and the fluid did exchange momentum


def test_no_drag_leaves_the_fluid_at_rest():
    x0, xd, t = _cell(amp=0.15, seed=4)
    s = oracle.System((14, 12, 12), 1.0, (0, 0, 0), (1, 0, 0))
    s.add_mesh(x0, t, MOD)
    s.set_nodes(0, xd)
    s.set_dynamics(0.8, 0.0)
    bare = oracle.System((14, 12, 12), 1.0, (0, 0, 0), (1, 0, 0))   # the same fluid, no cell
    c0 = xd.mean(axis=0)
    for _ in range(20):
        s.step(1)
        bare.step(1)
    assert np.array_equal(s.get_f(), bare.get_f())
    assert np.abs(s.nodes(0).mean(axis=0) - c0).max() < 1e-14
    assert np.abs(s.velocities(0).sum(axis=0)).max() < 1e-14
    assert np.abs(s.nodes(0) - xd).max() > 1e-3      # the cell does deform
    assert np.abs(s.nodes(0) - xd).max() < 1.0       # and stays bounded


def test_massless_limit_first_cycle():
    x0, xd, t = _cell(amp=0.15, seed=5)
    G = (1e-5, 0.0, 0.0)
    a = oracle.System((14, 12, 12), 1.0, G, (1, 0, 0))
    b = oracle.System((14, 12, 12), 1.0, G, (1, 0, 0))
    for s in (a, b):
        s.add_mesh(x0, t, MOD)
        s.set_nodes(0, xd)
    b.set_dynamics(1e-9, 1.0)
    a.step(1)
    b.step(1)
    fa, fb = a.get_f(), b.get_f()
    _, w, _ = oracle.constants()
    assert np.abs((fb - fa)).max() <= 1e-8 * np.abs(fa - w[:, None]).max()
    # U = 0 in the fluid at rest: the points move by F / gamma
    F = a.forces(0)
    assert np.abs(b.nodes(0) - xd - F / 1.0).max() <= 1e-8 * np.abs(F).max()
