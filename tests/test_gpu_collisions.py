"""Collision forces on the GPU (soft sphere between cells, beads and walls)
against the FP64 oracle, through the C ABI."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1110_0995_gb300 import scene

pytestmark = pytest.mark.gpu
REP = (0.01, 1.0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def _sim(sc):
    from paper_1110_0995_gb300 import lbibm

    return lbibm.Simulation.from_scene(sc)


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, float) - b) / np.linalg.norm(b))


def test_collision_forces_match_oracle():
    """Force-free membranes: the first step's node forces are the collision
    forces alone; two cells overlapping their cut-off, one near a bead, one
    near a y-wall and one across the periodic x boundary."""
    x, t = scene.icosphere(2)
    zero = (0.0, 0.0, 0.0, 0.0, 0.0)
    pos = [(6.0, 8.0, 8.0), (8.3, 8.4, 8.1), (12.0, 1.1, 8.0), (30.8, 8.0, 9.0), (1.2, 8.2, 9.1)]
    meshes = [scene.Mesh("rbc", scene.quantize(1.5 * x + np.array(p), scene.POS_QUANTUM), t, zero) for p in pos]
    spheres = np.array([[13.0, 3.5, 8.0, 1.5]], np.float32)
    sc = scene.Scene(name="collide", dims=(32, 16, 16), tau=1.0, periodic=(1, 0, 0), spheres=spheres,
                     meshes=meshes, repulsion=REP)
    sim = _sim(sc)
    ref = oracle.System.from_scene(sc)
    sim.step(1)
    ref.step(1)
    Fo = np.concatenate([ref.forces(m) for m in range(len(meshes))])
    F = np.concatenate([sim.forces(m) for m in range(len(meshes))])
    assert np.abs(Fo).max() > 1e-3
    assert np.abs(F - Fo).max() < 1e-5 * np.abs(Fo).max()


def test_small_filter_with_collisions():
    """96x48x32 filter, 4 red + 1 tumor cell, collisions on: 300 steps."""
    sc = dataclasses.replace(scene.small_filter(seed=5, steps=300), repulsion=REP)
    sim = _sim(sc)
    ref = oracle.System.from_scene(sc)
    sim.step(sc.steps)
    ref.step(sc.steps)
    assert rel_l2(sim.fields()[1], ref.fields()[1]) < 1e-5
    for m in range(len(sc.meshes)):
        assert np.abs(sim.nodes(m) - ref.nodes(m)).max() < 1e-5
    assert sim.diagnostics()[4] == 0
