"""Stiffness limit of the explicitly coupled, massless immersed-boundary cycle.

Pins the finding that sets the parity horizon and the workload moduli: with
the 642-node red-cell mesh (edges 0.3-0.7 lu) at tau = 1, the stated
stretching modulus ks = 0.05 makes perturbations of FP32 size grow (the oracle
run against itself from positions moved by 1e-8 lu exceeds 1e-5 in u after
1000 steps), while ks = 0.02 damps them.  This is a property of the method's
discretisation, measured on the FP64 oracle alone.
"""
import numpy as np
import pytest

import oracle
from paper_1110_0995_gb300 import scene


def _sensitivity(moduli, steps):
    sc = scene.channel_plain(seed=1, moduli=moduli)
    a = oracle.System.from_scene(sc)
    b = oracle.System.from_scene(sc)
    x0 = sc.meshes[0].rest
    b.set_nodes(0, x0 + 1e-8 * np.random.default_rng(0).standard_normal(x0.shape))
    out = []
    for n in steps:
        a.step(n)
        b.step(n)
        _, ua = a.fields()
        _, ub = b.fields()
        out.append(np.linalg.norm(ua - ub) / np.linalg.norm(ua))
    return out


@pytest.mark.slow
def test_stated_stretching_modulus_amplifies_perturbations():
    s = _sensitivity(scene.SPEC, [400, 600])
    assert s[0] < 1e-5 < s[1]


@pytest.mark.slow
def test_stable_stretching_modulus_damps_perturbations():
    s = _sensitivity(scene.STABLE, [500, 500])
    assert s[1] < s[0] < 1e-7


def _tumor_cell_at_rest(moduli, blocks=6, every=500):
    """max |u| every `every` steps of a tumor cell (2562-node mesh, radius 8)
    at rest in a still fluid, its nodes moved by 1e-6 lu."""
    v, t = scene.cell_template("ctc")
    rest = scene.quantize(v + np.array([19.5, 15.5, 15.5]), scene.POS_QUANTUM)
    sc = scene.Scene(name="ctc_rest", dims=(40, 32, 32), tau=1.0, body_force=(0, 0, 0), periodic=(1, 0, 0),
                     meshes=[scene.Mesh("ctc", rest, t, moduli)], steps=0)
    s = oracle.System.from_scene(sc)
    s.set_nodes(0, rest + 1e-6 * np.random.default_rng(0).standard_normal(rest.shape))
    out = []
    for _ in range(blocks):
        s.step(every)
        _, u = s.fields()
        out.append(np.abs(u).max())
    return out


@pytest.mark.slow
def test_tumor_cell_mesh_grows_at_ks_0_03_and_damps_at_0_003():
    """The 2562-node tumor-cell mesh (edges ~0.6 lu) has a mode that the
    explicit cycle amplifies at ks = 0.03, kb = kal = 0.01 (x5 per 500 steps
    once it dominates), and damps at ks = kb = kal = 0.003, the workloads'
    tumor-cell set."""
    grow = _tumor_cell_at_rest((0.03, 0.01, 0.01, 0.5, 0.9))
    assert grow[5] > 20 * grow[3] and grow[5] > 1e-6
    soft = _tumor_cell_at_rest((0.003, 0.003, 0.003, 0.5, 0.9))
    assert soft[5] < soft[1] < 2e-8
