"""Writes tests/golden/adjoint_reference_128x64x64.json: the FP64 oracle's
gradient of the adjoint workload's objective, for the GPU adjoint test.

Workload: the 128x64x64 channel with two posts of six differentiable
(Brinkman) beads, one tumor cell (the objective cell, mesh 0) and eight red
cells, 400 cycles (scene.adjoint_channel).  J = mean x displacement of the
tumor cell's nodes after the 400 cycles.  For each of the 36 bead-centre
coordinates and the tumor cell's ks and kb: dJ/dp from one forward pass of the
oracle in FP64 dual numbers (forward mode, one parameter per pass), and for the
largest bead component and ks a central finite difference of J with h = 1e-4
(two plain FP64 runs each), which checks the dual numbers independently.

Calls only the oracle (and the seeded scene generator).  Run from the
repository root:  python tests/golden/make_adjoint_reference.py   (~40 min on
8 cores: 38 dual passes and 4 plain runs of 400 cycles on 524,288 nodes).
"""
import dataclasses
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1110_0995_gb300 import scene  # noqa: E402

STEPS = 400
H = 1e-4
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "adjoint_reference_128x64x64.json")


def main():
    sc = scene.adjoint_channel(steps=STEPS)
    t0 = time.time()
    ref = oracle.DiffProblem.from_scene(sc)
    J = ref.run(STEPS, 0)
    grads = {"beads": [], "ks": None, "kb": None}
    for i in range(3 * len(sc.spheres)):
        _, d = ref.run(STEPS, 0, ("bead", i))
        grads["beads"].append(d)
        print(f"bead {i // 3} axis {i % 3}: {d:.9e}  ({time.time() - t0:.0f} s)", flush=True)
    for name in ("ks", "kb"):
        _, grads[name] = ref.run(STEPS, 0, (name,))
        print(f"{name}: {grads[name]:.9e}", flush=True)
    # central differences of the plain FP64 objective
    fd = {}
    ib = int(np.argmax(np.abs(grads["beads"])))
    for tag in (f"bead_{ib}", "ks"):
        vals = []
        for sgn in (1.0, -1.0):
            if tag == "ks":
                mods = [m.moduli for m in sc.meshes]
                mods[0] = (mods[0][0] + sgn * H,) + tuple(mods[0][1:])
                p = oracle.DiffProblem.from_scene(sc, moduli=mods)
            else:
                sph = np.asarray(sc.spheres, np.float64).copy()
                sph[ib // 3, ib % 3] += sgn * H
                p = oracle.DiffProblem.from_scene(dataclasses.replace(sc, spheres=sph))
            vals.append(p.run(STEPS, 0))
        fd[tag] = (vals[0] - vals[1]) / (2 * H)
        print(f"FD {tag}: {fd[tag]:.9e}", flush=True)
    out = {"workload": "scene.adjoint_channel(seed=41): 128x64x64, 12 Brinkman beads (alpha 2, delta 0.5), "
                       "1 tumor cell (objective, mesh 0) + 8 red cells",
           "steps": STEPS, "J": J, "dJ_dbeads": grads["beads"], "dJ_dks": grads["ks"], "dJ_dkb": grads["kb"],
           "fd_h": H, "fd": fd, "how": "FP64 oracle: forward-mode dual numbers, one parameter per pass; "
                                      "central differences of plain FP64 runs for two parameters"}
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", OUT, f"({time.time() - t0:.0f} s)")


if __name__ == "__main__":
    main()
