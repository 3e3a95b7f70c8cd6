"""Pins of the oracle's magnetic bead interaction (Sec. 2.5: the force of
bead 1 on bead 2 for moments m1, m2 at separation r = x2 - x1, printed with
an unbalanced bracket that is closed after its last term), the contact force
and the overdamped bead motion.

* two moments along their separation attract with 6 c m^2 / r^4 and two
  moments across it repel with 3 c m^2 / r^4 (the textbook dipole results);
* the force is minus the gradient (with respect to x2) of the separately
  written pair energy c / r^3 [m1.m2 - 3 (m1.r)(m2.r) / r^2], by central
  differences, for random moments and separations;
* Newton's third law pair by pair, and zero total force for N beads;
* a pair across a periodic boundary acts as through the minimum image;
* two beads along the field relax to the separation where the dipole
  attraction equals the contact force k (2R - d) (root found independently).
"""
import numpy as np
import pytest

import oracle


def test_axial_attraction_and_transverse_repulsion():
    c, m, r = 0.7, 1.3, 2.5
    F = oracle.dipole_force([0, 0, m], [0, 0, m], [0, 0, r], c)
    assert F == pytest.approx([0, 0, -6 * c * m * m / r**4], abs=1e-16)
    F = oracle.dipole_force([0, 0, m], [0, 0, m], [r, 0, 0], c)
    assert F == pytest.approx([3 * c * m * m / r**4, 0, 0], abs=1e-16)


@pytest.mark.parametrize("seed", range(5))
def test_force_is_minus_energy_gradient(seed):
    rng = np.random.default_rng(seed)
    m1, m2 = rng.normal(size=3), rng.normal(size=3)
    r = rng.normal(size=3)
    r *= (1.5 + rng.random()) / np.linalg.norm(r)
    c = 0.9
    F = oracle.dipole_force(m1, m2, r, c)
    h = 1e-5
    g = np.zeros(3)
    for d in range(3):
        e = np.zeros(3)
        e[d] = h
        g[d] = (oracle.dipole_energy(m1, m2, r + e, c) - oracle.dipole_energy(m1, m2, r - e, c)) / (2 * h)
    assert np.abs(F + g).max() <= 1e-8 * np.abs(F).max()


def test_third_law_and_zero_total():
    rng = np.random.default_rng(11)
    m1, m2 = rng.normal(size=3), rng.normal(size=3)
    r = np.array([0.7, -1.9, 1.1])
    F12 = oracle.dipole_force(m1, m2, r, 1.0)
    F21 = oracle.dipole_force(m2, m1, -r, 1.0)
    assert np.abs(F12 + F21).max() < 1e-15
    n = 12
    x = rng.uniform(0, 6, size=(n, 3))
    m = np.tile([0.0, 0.0, 1.0], (n, 1)) + 0.1 * rng.normal(size=(n, 3))
    F = oracle.bead_forces(x, m, 1.0, 0.8, 5.0)
    assert np.abs(F.sum(axis=0)).max() <= 1e-12 * np.abs(F).max()
    assert np.abs(F).max() > 0


def test_minimum_image_across_a_periodic_boundary():
    m = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 1.0]])
    box = (10.0, 10.0, 10.0)
    near = oracle.bead_forces([[5.0, 5.0, 9.5], [5.0, 5.0, 0.5]], m, 1.0, 0.4, 1.0, box, (0, 0, 1))
    direct = oracle.bead_forces([[5.0, 5.0, 4.5], [5.0, 5.0, 5.5]], m, 1.0, 0.4, 1.0, box, (0, 0, 0))
    assert np.abs(near - direct).max() < 1e-15


def test_pair_relaxes_to_force_balance():
    c, m, R, k = 1.0, 1.0, 1.0, 10.0
    # d* solves 6 c m^2 / d^4 = k (2R - d): bisection on the separately written balance
    lo, hi = 1.0, 2.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if 6 * c * m * m / mid**4 - k * (2 * R - mid) > 0:   # net attraction: the balance lies closer
            hi = mid
        else:
            lo = mid
    d_star = 0.5 * (lo + hi)
    x = oracle.bead_relax([[0.0, 0.0, 0.0], [0.0, 0.0, 3.0]], [[0, 0, m], [0, 0, m]], c, R, k,
                          mobility=1.0, dt=0.02, steps=3000)
    assert x[1, 2] - x[0, 2] == pytest.approx(d_star, abs=1e-10)
    assert np.abs(x[:, :2]).max() == 0.0
    assert x[0, 2] + x[1, 2] == pytest.approx(3.0, abs=1e-12)   # symmetric motion
