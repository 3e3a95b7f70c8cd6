"""The allocation-free area/volume entry point against the context's own.

ibm_area_volume_noalloc serves callers that cannot allocate device memory
(frameworks that own the device memory pool, latency-critical loops that cannot
afford cudaMalloc's synchronisation, fixed-budget embedded callers): its scratch
is a fixed device array inside the library.  This test calls it through the C
ABI on caller-owned device buffers, twice in a row with different node
positions (the second call reuses the scratch the first one left behind), and
checks both results against ibm_get_area_volume of a context holding the same
meshes at the same positions, with the tolerance of the other area / volume
parity tests (2e-8 of the rest value plus 1e-5 of the change).  It lives in a
file of its own so that it runs after every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1110_0995_gb300 import scene

pytestmark = pytest.mark.gpu


def _meshes():
    out = []
    for kind, shift in (("rbc", (10.0, 12.0, 9.0)), ("ctc", (30.0, 15.0, 16.0)), ("rbc", (22.0, 6.0, 7.0))):
        v, t = scene.cell_template(kind)
        out.append(scene.Mesh(kind, scene.quantize(v + np.array(shift), scene.POS_QUANTUM), t, scene.STABLE[kind]))
    return out


def _deformed(meshes, seed, amp):
    rng = np.random.default_rng(seed)
    return [scene.quantize(m.rest + amp * rng.standard_normal(m.rest.shape), scene.POS_QUANTUM) for m in meshes]


def _context_area_volume(meshes, positions):
    from paper_1110_0995_gb300 import lbibm

    sc = scene.Scene(name="noalloc", dims=(48, 32, 32), periodic=(1, 1, 1), meshes=meshes)
    sim = lbibm.Simulation.from_scene(sc)
    for k, x in enumerate(positions):
        sim.set_nodes(k, x)
    S, V = sim.area_volume()
    sim.close()
    return S, V


def _noalloc_area_volume(meshes, positions):
    import torch

    from paper_1110_0995_gb300 import lbibm

    L = lbibm.lib()
    xyz = np.concatenate(positions).astype(np.float64)
    tris, starts, base = [], [0], 0
    for m in meshes:
        tris.append(m.tris.astype(np.int64) + base)
        base += m.n_nodes
        starts.append(starts[-1] + m.n_tris)
    tris = np.concatenate(tris).astype(np.int32)
    starts = np.asarray(starts, dtype=np.int32)
    dev = torch.device("cuda:0")
    d_xyz = torch.from_numpy(xyz).to(dev)
    d_tris = torch.from_numpy(tris).to(dev)
    d_starts = torch.from_numpy(starts).to(dev)
    d_area = torch.full((len(meshes),), float("nan"), dtype=torch.float64, device=dev)
    d_vol = torch.full((len(meshes),), float("nan"), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    st = L.ibm_area_volume_noalloc(ctypes.c_void_p(d_xyz.data_ptr()), ctypes.c_void_p(d_tris.data_ptr()),
                                   ctypes.c_void_p(d_starts.data_ptr()), starts.ctypes.data_as(ctypes.c_void_p),
                                   len(meshes), ctypes.c_void_p(d_area.data_ptr()), ctypes.c_void_p(d_vol.data_ptr()),
                                   ctypes.c_void_p(stream.cuda_stream))
    assert st == lbibm.LB_OK
    torch.cuda.synchronize(dev)
    return d_area.cpu().numpy(), d_vol.cpu().numpy()


def test_noalloc_area_volume_matches_context_two_calls():
    import __graft_entry__

    __graft_entry__.build()
    meshes = _meshes()
    S0 = np.array([0.5 * np.linalg.norm(np.cross(m.rest[m.tris[:, 1]] - m.rest[m.tris[:, 0]],
                                                 m.rest[m.tris[:, 2]] - m.rest[m.tris[:, 0]]), axis=1).sum()
                   for m in meshes])
    V0 = np.array([np.linalg.det(np.stack([m.rest[m.tris[:, k]] for k in range(3)], axis=1)).sum() / 6
                   for m in meshes])
    for call, (seed, amp) in enumerate([(1, 0.03), (2, 0.08)]):
        pos = _deformed(meshes, seed, amp)
        S, V = _noalloc_area_volume(meshes, pos)
        Sc, Vc = _context_area_volume(meshes, pos)
        assert np.abs(S - Sc).max() <= (2e-8 * S0 + 1e-5 * np.abs(Sc - S0)).max(), (call, S, Sc)
        assert np.abs(V - Vc).max() <= (2e-8 * V0 + 1e-5 * np.abs(Vc - V0)).max(), (call, V, Vc)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_1110_0995_gb300 import lbibm

    L = lbibm.lib()
    # 1,000 cells, the largest with 66 chunks of 256 triangles: 66,000 partials > 65,536.
    # The size check runs on the host before any device work, so the device
    # pointers are never touched.
    counts = np.ones(1000, dtype=np.int64)
    counts[0] = 66 * 256
    starts = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    dummy = ctypes.c_void_p(1)
    st = L.ibm_area_volume_noalloc(dummy, dummy, dummy, starts.ctypes.data_as(ctypes.c_void_p), 1000,
                                   dummy, dummy, None)
    assert st == lbibm.LB_ERR_ARG
    # more cells than the grid allows
    starts = np.arange(70001, dtype=np.int32)
    st = L.ibm_area_volume_noalloc(dummy, dummy, dummy, starts.ctypes.data_as(ctypes.c_void_p), 70000,
                                   dummy, dummy, None)
    assert st == lbibm.LB_ERR_ARG
