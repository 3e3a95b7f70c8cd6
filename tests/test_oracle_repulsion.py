"""Pins of the oracle's collision forces (Sec. 2.4 reading: harmonic soft
sphere k (d_c - d) below separation d_c between nodes of different cells,
between a node and a bead surface, between a node and a wall).

Checked against what the mathematics fixes, with force-free membranes so the
last step's node forces are the collision forces alone:
* they are minus the gradient of the potential sum (k/2)(d_c - d)^2, whose
  value is computed here independently, by central differences in the node
  positions;
* node-node forces conserve momentum and angular momentum (central, pairwise);
* nothing acts beyond d_c, and across the periodic x boundary the nearest image
  interacts.
"""
import numpy as np
import pytest

import oracle
from paper_1110_0995_gb300 import scene

ZERO = (0.0, 0.0, 0.0, 0.0, 0.0)   # force-free membranes
K, DC = 0.013, 0.9


def _two_cells(shift, dims=(20, 12, 12), per=(1, 0, 0)):
    x, t = scene.icosphere(0)
    a = 0.45 * x + np.array([6.0, 6.0, 6.0])
    b = 0.45 * x + np.array([6.0, 6.0, 6.0]) + np.asarray(shift, float)
    return a, b, t, dims, per


def _forces(cells, t, dims, per, spheres=np.zeros((0, 4))):
    s = oracle.System(dims, 1.0, (0, 0, 0), per)
    for c in cells:
        s.add_mesh(c, t, ZERO)
    s.set_repulsion(K, DC, spheres)
    s.step(1)
    return [s.forces(m) for m in range(len(cells))]


def _energy(cells, dims, per, spheres=np.zeros((0, 4))):
    E = 0.0
    for i in range(len(cells)):
        for j in range(i + 1, len(cells)):
            d = cells[i][:, None, :] - cells[j][None, :, :]
            for ax in range(3):
                if per[ax]:
                    d[..., ax] -= dims[ax] * np.round(d[..., ax] / dims[ax])
            r = np.sqrt((d ** 2).sum(-1))
            E += 0.5 * K * ((DC - r[r < DC]) ** 2).sum()
    for c in cells:
        for sp in spheres:
            g = np.sqrt(((c - sp[:3]) ** 2).sum(-1)) - sp[3]
            E += 0.5 * K * ((DC - g[g < DC]) ** 2).sum()
        for ax in range(3):
            if not per[ax]:
                for gap in (c[:, ax] + 0.5, dims[ax] - 0.5 - c[:, ax]):
                    E += 0.5 * K * ((DC - gap[gap < DC]) ** 2).sum()
    return E


def _fd_check(cells, t, dims, per, spheres=np.zeros((0, 4))):
    F = _forces(cells, t, dims, per, spheres)
    h = 1e-6
    rng = np.random.default_rng(0)
    for _ in range(12):
        m = rng.integers(len(cells))
        j = rng.integers(cells[m].shape[0])
        ax = rng.integers(3)
        cp = [c.copy() for c in cells]
        cm = [c.copy() for c in cells]
        cp[m][j, ax] += h
        cm[m][j, ax] -= h
        fd = -(_energy(cp, dims, per, spheres) - _energy(cm, dims, per, spheres)) / (2 * h)
        assert F[m][j, ax] == pytest.approx(fd, rel=1e-6, abs=1e-12)
    return F


def test_cell_cell_gradient_and_conservation():
    a, b, t, dims, per = _two_cells((0.95, 0.1, -0.05))
    F = _fd_check([a, b], t, dims, per)
    assert np.abs(F[0]).max() > 1e-3
    tot = F[0].sum(0) + F[1].sum(0)
    assert np.abs(tot).max() < 1e-15
    L = np.cross(a, F[0]).sum(0) + np.cross(b, F[1]).sum(0)
    assert np.abs(L).max() < 1e-14


def test_cut_off_and_periodic_image():
    a, b, t, dims, per = _two_cells((0.45 * 2 + DC + 0.01, 0, 0))   # nearest nodes just beyond d_c
    F = _forces([a, b], t, dims, per)
    assert np.abs(F[0]).max() == 0.0 and np.abs(F[1]).max() == 0.0
    a, b, t, dims, per = _two_cells((20 - 1.0, 0, 0))               # close only through x periodicity
    F = _fd_check([a, b], t, dims, per)
    # b sits 1 lu to the left of a through the boundary: a is pushed to +x
    assert F[0][:, 0].sum() > 0 and abs(F[0].sum(0) + F[1].sum(0)).max() < 1e-15


def test_bead_and_wall_gradient():
    x, t = scene.icosphere(0)
    c = 0.45 * x + np.array([6.0, 0.6, 11.0])      # near the y-low and z-high walls
    beads = np.array([[7.1, 1.0, 11.2, 0.5]])
    F = _fd_check([c], t, (20, 12, 12), (1, 0, 0), beads)
    assert F[0][:, 1].max() > 0 and F[0][:, 2].min() < 0
