"""PyTorch autograd entry for the filter objective of the differentiable variant.

``filter_objective(beads, ks, kb, scene, steps)`` returns J, the x
displacement of the scene's objective cell (mesh 0) after ``steps`` cycles,
as a differentiable function of the bead centres (n x 3) and of that cell's
stretching / bending moduli.  The forward builds a simulation with the given
parameters (beads as the smooth Brinkman solid fraction, see
``lb_set_brinkman``) and runs ``lb_adjoint`` once: J and every gradient come
from that one call (checkpointed forward + reverse sweep on the GPU), and
``backward`` only scales the stored gradients by the incoming one.  Torch is
used for the tensors and the autograd graph; every step runs in the library.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import lbibm


class FilterObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, beads, ks, kb, scene, steps: int, ckpt_every: int = 50, alpha: float = 2.0,
                delta: float = 0.5):
        b = beads.detach().to("cpu", torch.float64).numpy().reshape(-1, 3)
        radii = np.asarray(scene.spheres, np.float64).reshape(-1, 4)[:, 3]
        if len(radii) != len(b):
            raise ValueError("one centre per bead of the scene")
        meshes = list(scene.meshes)
        m0 = meshes[0]
        meshes[0] = dataclasses.replace(m0, moduli=(float(ks), float(kb)) + tuple(m0.moduli[2:]))
        bare = dataclasses.replace(scene, spheres=np.zeros((0, 4), np.float32), meshes=meshes)
        sim = lbibm.Simulation.from_scene(bare)
        try:
            sim.set_brinkman(np.column_stack([b, radii]), alpha, delta)
            r = sim.adjoint(int(steps), int(ckpt_every), 0)
        finally:
            sim.close()
        dev, dt = beads.device, beads.dtype
        ctx.save_for_backward(torch.as_tensor(r["beads"], dtype=dt, device=dev).reshape(beads.shape),
                              torch.tensor(r["ks"], dtype=dt, device=dev), torch.tensor(r["kb"], dtype=dt, device=dev))
        return torch.tensor(r["J"], dtype=dt, device=dev)

    @staticmethod
    def backward(ctx, gJ):
        g_beads, g_ks, g_kb = ctx.saved_tensors
        return gJ * g_beads, gJ * g_ks, gJ * g_kb, None, None, None, None, None


def filter_objective(beads: torch.Tensor, ks: torch.Tensor, kb: torch.Tensor, scene, steps: int,
                     ckpt_every: int = 50) -> torch.Tensor:
    """J(beads, ks, kb) with gradients by the library's discrete adjoint."""
    return FilterObjective.apply(beads, ks, kb, scene, steps, ckpt_every)
