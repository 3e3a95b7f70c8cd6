"""Out-of-bounds device writes, checked without a memory checker: every
device allocation of the contexts created here carries 64 KiB of a fixed byte
pattern before and after it (lb_set_guard_zones), and after each workload no
byte of any guard zone may have changed.  Workloads: every stream-collide
variant of both storages on ragged lattices with walls, a moving wall and
obstacles (the TMA-staged variant on its lattices), the small filter with
cells (sequential, deterministic, overlapped schedule, points with mass,
collisions, 16-bit storage), a batch of channels of uneven size and the
adjoint.  A self test first shows that the count sees a changed byte in every
zone."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_1110_0995_gb300 import scene

pytestmark = pytest.mark.gpu

GUARD = 64 * 1024


@pytest.fixture(scope="module", autouse=True)
def _guards():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1110_0995_gb300 import lbibm

    lbibm.set_guard_zones(GUARD)
    yield
    lbibm.set_guard_zones(0)     # contexts of later tests without guard zones


def _sim(sc, storage="f32"):
    from paper_1110_0995_gb300 import lbibm

    return lbibm.Simulation.from_scene(sc, storage=storage)


def _ragged(dims, periodic=(1, 0, 1), wall=((0, 0, 0), (0.02, 0, 0.01))):
    sph = np.array([[9.0, 11.5, 8.25, 3.0], [25.5, 6.0, 12.0, 2.5], [30.0, 17.0, 3.0, 2.0]], np.float32)
    sph = scene.quantize(sph * np.array([dims[0] / 37, dims[1] / 23, dims[2] / 19, 1.0]),
                         scene.SPHERE_QUANTUM).astype(np.float32)
    return scene.Scene(name="ragged", dims=dims, tau=0.8, body_force=(2e-5, -1e-5, 5e-6), periodic=periodic,
                       wall_velocity=wall, spheres=sph, meshes=[], steps=0)


def _run_and_check(sim, steps):
    sim.step(steps)
    assert sim.diagnostics()[4] == 0
    assert sim.guard_damage() == 0


def test_self_test_sees_every_zone():
    sim = _sim(scene.small_filter(seed=5, steps=0))
    n_alloc = sim.guard_damage(self_test=True)
    assert n_alloc > 0 and n_alloc % 2 == 0
    assert sim.guard_damage() == 0          # restored


@pytest.mark.parametrize("storage,variants", [
    ("f32", [(-1, 128), (-1, 256), (0, 256), (1, 128), (1, 256), (2, 128), (2, 256), (4, 128), (4, 256)]),
    ("f16", [(-1, 128), (0, 256), (1, 128), (1, 256), (2, 128), (2, 256), (4, 64), (4, 128)]),
    ("bf16", [(1, 128), (2, 128), (4, 64)])])
def test_every_variant_writes_inside_its_arrays(storage, variants):
    from paper_1110_0995_gb300 import lbibm

    for dims in ((36, 23, 19), (64, 24, 19)):
        for v in variants:
            sim = _sim(_ragged(dims), storage)
            try:
                sim.set_kernel_config(*v)
            except lbibm.LbError:
                continue                       # variant not offered on this lattice
            sim.set_prefetch(65536 if v[0] > 0 else 0)
            _run_and_check(sim, 25)


@pytest.mark.parametrize("tile", [256, 512])
def test_tma_variant_writes_inside_its_arrays(tile):
    sim = _sim(_ragged((64, 24, 19), periodic=(1, 0, 0)))
    sim.set_kernel_config(-2, tile)
    _run_and_check(sim, 25)


@pytest.mark.parametrize("mode", ["default", "deterministic", "overlapped", "massive", "collisions", "f16", "bf16"])
def test_filter_cycle_writes_inside_its_arrays(mode):
    sc = scene.small_filter(seed=5, steps=0)
    storage = mode if mode in ("f16", "bf16") else "f32"
    if mode == "massive":
        sc = dataclasses.replace(sc, ib_dynamics=(0.05, 5.0))
    if mode == "collisions":
        sc = dataclasses.replace(sc, repulsion=(0.01, 1.0))
    sim = _sim(sc, storage)
    if mode == "deterministic":
        sim.set_deterministic(True)
    if mode == "overlapped":
        sim.set_schedule(1)
    _run_and_check(sim, 60)
    state = sim.save_state()
    sim.load_state(state)
    _run_and_check(sim, 10)


def test_batch_and_adjoint_write_inside_their_arrays():
    from paper_1110_0995_gb300 import lbibm

    scs = [scene.channel_plain(seed=s, steps=0, dims=d, moduli=scene.STABLE)
           for s, d in ((1, (32, 16, 64)), (2, (48, 24, 32)), (3, (40, 32, 24)))]
    sim = lbibm.Simulation.from_scenes(scs)
    _run_and_check(sim, 40)
    sc = scene.adjoint_channel_small(steps=20)
    bare = dataclasses.replace(sc, spheres=np.zeros((0, 4), np.float32))
    sim = lbibm.Simulation.from_scene(bare)
    sim.set_brinkman(np.asarray(sc.spheres, np.float64))
    sim.adjoint(20, ckpt_every=10)
    assert sim.guard_damage() == 0
