"""Shifted 16-bit population storage at the 512x256x128 filter scale (404
cells, 672 beads): error of FP32, FP16 and BF16 storage against the FP64
oracle per field after 200 cycles (rho, u, node positions, per-cell volume
change).

The 16-bit stores round stochastically (an unbiased rounding whose random bits
are a hash of the node and its moments).  Rounding to nearest gave every node
of a region of nearly uniform flow the same error, and those errors added up
over the cycles into a velocity error that viscosity does not damp: on GB300
FP16 reached 1.26e-3 and BF16 9.9e-3 in u with round-to-nearest, against
2.0e-4 and 1.6e-3 with stochastic rounding.  FP32 is held to the parity
tolerance, FP16 to the 1e-3 velocity target, BF16 (8-bit mantissa, reported,
not a target) to a regression bound of 3e-3."""
import numpy as np
import pytest

import oracle
from paper_1110_0995_gb300 import scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, float) - b) / np.linalg.norm(b))


def test_storage_precision_large_filter():
    from paper_1110_0995_gb300 import lbibm

    T = 200
    sc = scene.micropost_filter_large(seed=31, steps=T)
    ref = oracle.System.from_scene(sc)
    ref.step(T)
    rho_o, u_o = ref.fields()
    x_o = np.concatenate([ref.nodes(m) for m in range(len(sc.meshes))])
    V_o = np.array([oracle.mesh_area_volume(ref.nodes(m), sc.meshes[m].tris)[1] for m in range(len(sc.meshes))])
    V_0 = np.array([oracle.mesh_area_volume(m.rest, m.tris)[1] for m in sc.meshes])
    fluid = ref.solid if hasattr(ref, "solid") else None
    errs = {}
    for st in ("f32", "f16", "bf16"):
        sim = lbibm.Simulation.from_scene(sc, storage=st)
        sim.step(T)
        rho, u = sim.fields()
        x = np.zeros_like(x_o)
        sim.all_nodes_into(x)
        _, V = sim.area_volume()
        m = fluid == 0 if fluid is not None else slice(None)
        errs[st] = {
            "rho_max": float(np.abs(rho - rho_o)[m].max()),
            "u_rel_l2": rel_l2(u, u_o),
            "x_max": float(np.abs(x - x_o).max()),
            "dV_rel": float(np.abs((V - V_0) - (V_o - V_0)).max() / np.abs(V_o - V_0).max()),
        }
        print(st, errs[st])
        sim.close()
    assert errs["f32"]["u_rel_l2"] < 1e-5 and errs["f32"]["x_max"] < 1e-5
    assert errs["f16"]["u_rel_l2"] <= 1e-3
    assert errs["bf16"]["u_rel_l2"] <= 3e-3
