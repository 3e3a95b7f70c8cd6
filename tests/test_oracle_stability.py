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
