"""Pins of the oracle's differentiable variant (Brinkman beads) and of its
dual-number reference gradient, which the GPU adjoint is checked against.

* dual-number derivatives of J equal FP64 central finite differences of the
  same run (bead coordinates, ks, kb of the objective cell), Richardson-
  extrapolated: with h small enough to hide the O(h^2) term the differences
  drown in the run's own rounding (~1e-15 in J);
* with no beads (phi = 0) the variant reproduces the plain coupled cycle;
* inside a bead (phi = 1, alpha = 2) a uniformly forced periodic box settles
  at u = g / 2 exactly (the implicit Brinkman closed form);
* phi = 1/2 on a lone bead's surface, -> 1 at its centre, -> 0 far away, and
  the union of two beads is 1 - (1 - phi_1)(1 - phi_2).
"""
import numpy as np
import pytest

import oracle
from paper_1110_0995_gb300 import scene


def _tiny(beads=((12.0, 5.0, 8.0, 2.5), (12.5, 11.0, 8.0, 2.0)), G=(2e-4, 0.0, 0.0)):
    x, t = scene.icosphere(1)
    x0 = 2.2 * x + np.array([5.3, 8.1, 7.9])
    p = oracle.DiffProblem((24, 16, 16), 1.0, G, (1, 0, 0), np.array(beads, float))
    p.add_mesh(x0, t, (0.02, 0.01, 0.01, 0.5, 0.9))
    return p, x0, t


@pytest.mark.parametrize("seed", [("bead", 0), ("bead", 1), ("bead", 4), ("ks",), ("kb",)])
def test_dual_derivative_matches_central_differences(seed):
    steps = 12
    p, x0, t = _tiny()
    J, dJ = p.run(steps, 0, seed)
    h = 1e-2 if seed[0] == "bead" else 1e-3

    def J_at(delta):
        beads = np.array(((12.0, 5.0, 8.0, 2.5), (12.5, 11.0, 8.0, 2.0)))
        mod = np.array((0.02, 0.01, 0.01, 0.5, 0.9))
        if seed[0] == "bead":
            beads[seed[1] // 3, seed[1] % 3] += delta
        elif seed[0] == "ks":
            mod[0] += delta
        else:
            mod[1] += delta
        q = oracle.DiffProblem((24, 16, 16), 1.0, (2e-4, 0.0, 0.0), (1, 0, 0), beads)
        q.add_mesh(x0, t, mod)
        return q.run(steps, 0)

    def central(hh):
        return (J_at(hh) - J_at(-hh)) / (2 * hh)

    fd = (4 * central(h) - central(2 * h)) / 3
    assert J == pytest.approx(p.run(steps, 0), rel=1e-15, abs=1e-18)
    assert abs(dJ) > 0
    assert dJ == pytest.approx(fd, rel=5e-5)


def test_no_beads_reproduces_plain_cycle():
    x, t = scene.icosphere(1)
    x0 = 2.2 * x + np.array([5.3, 8.1, 7.9])
    mod = (0.02, 0.01, 0.01, 0.5, 0.9)
    p = oracle.DiffProblem((16, 12, 12), 1.0, (2e-4, 0, 0), (1, 0, 0), np.zeros((0, 4)))
    p.add_mesh(x0, t, mod)
    _, u, xs = p.state(15, 0)
    s = oracle.System((16, 12, 12), 1.0, (2e-4, 0, 0), (1, 0, 0))
    s.add_mesh(x0, t, mod)
    s.step(15)
    _, uo = s.fields()
    assert np.abs(u - uo).max() < 1e-15
    assert np.abs(xs - s.nodes(0)).max() < 1e-13


def test_solid_box_holds_half_the_force():
    G = np.array([3e-4, -1e-4, 2e-4])
    p = oracle.DiffProblem((6, 5, 4), 1.0, G, (1, 1, 1), np.array([[3.0, 2.5, 2.0, 1000.0]]))
    x, t = scene.icosphere(0)
    p.add_mesh(0.5 * x + 2.5, t, (0.0, 0.0, 0.0, 0.0, 0.0))   # force-free mesh
    assert np.all(p.phi() == 1.0)
    _, u, _ = p.state(5, 0)
    assert np.abs(u - (G / 2)[:, None]).max() < 1e-15


def test_phi_single_and_union():
    p = oracle.DiffProblem((20, 20, 20), 1.0, (0, 0, 0), (1, 1, 1), np.array([[10.0, 10.0, 10.0, 4.0]]), delta=0.5)
    phi = p.phi().reshape(20, 20, 20)   # [z, y, x]
    assert phi[10, 10, 14] == pytest.approx(0.5, abs=1e-15)       # on the surface
    assert phi[10, 10, 10] == pytest.approx(1.0, abs=1e-6)        # centre: 1/2 (1 + tanh 8)
    assert phi[10, 10, 19] < 1e-7                                  # 5 lu outside
    q = oracle.DiffProblem((20, 20, 20), 1.0, (0, 0, 0), (1, 1, 1),
                           np.array([[10.0, 10.0, 10.0, 4.0], [13.0, 10.0, 10.0, 3.0]]), delta=0.5)
    r = oracle.DiffProblem((20, 20, 20), 1.0, (0, 0, 0), (1, 1, 1), np.array([[13.0, 10.0, 10.0, 3.0]]), delta=0.5)
    assert np.abs(q.phi() - (1 - (1 - p.phi()) * (1 - r.phi()))).max() < 1e-15
