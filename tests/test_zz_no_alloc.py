"""The allocation-free area/volume entry point against the FP64 oracle and
against the context's own reduction.

ibm_area_volume_noalloc serves callers that cannot allocate device memory
(frameworks that own the device memory pool, latency-critical loops that cannot
afford cudaMalloc's synchronisation, fixed-budget embedded callers): its scratch
is a fixed device array inside the library.  This test calls it through the C
ABI on caller-owned device buffers, twice in a row with different node
positions (the second call reuses the scratch the first one left behind), with
a cell that owns no triangle between the meshes, and checks both results
against the oracle's FP64 area and volume of every mesh (both sides FP64, only
the summation order differs: 1e-10 relative) and against ibm_get_area_volume
of a context holding the same meshes at the same positions, with the tolerance
of the other area / volume parity tests (2e-8 of the rest value plus 1e-5 of
the change).  A call with no cell returns LB_OK and touches nothing.  It lives
in a file of its own so that it runs after every other test.
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


def _noalloc_area_volume(meshes, positions, empty_after=None):
    """Areas and volumes of the meshes through the C ABI; with empty_after = k a
    cell owning no triangle is inserted after mesh k (its area and volume are
    returned separately)."""
    import torch

    from paper_1110_0995_gb300 import lbibm

    L = lbibm.lib()
    xyz = np.concatenate(positions).astype(np.float64)
    tris, starts, base = [], [0], 0
    for k, m in enumerate(meshes):
        tris.append(m.tris.astype(np.int64) + base)
        base += m.n_nodes
        starts.append(starts[-1] + m.n_tris)
        if empty_after == k:
            starts.append(starts[-1])
    tris = np.concatenate(tris).astype(np.int32)
    starts = np.asarray(starts, dtype=np.int32)
    n_cells = len(starts) - 1
    dev = torch.device("cuda:0")
    d_xyz = torch.from_numpy(xyz).to(dev)
    d_tris = torch.from_numpy(tris).to(dev)
    d_starts = torch.from_numpy(starts).to(dev)
    d_area = torch.full((n_cells,), float("nan"), dtype=torch.float64, device=dev)
    d_vol = torch.full((n_cells,), float("nan"), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    st = L.ibm_area_volume_noalloc(ctypes.c_void_p(d_xyz.data_ptr()), ctypes.c_void_p(d_tris.data_ptr()),
                                   ctypes.c_void_p(d_starts.data_ptr()), starts.ctypes.data_as(ctypes.c_void_p),
                                   n_cells, ctypes.c_void_p(d_area.data_ptr()), ctypes.c_void_p(d_vol.data_ptr()),
                                   ctypes.c_void_p(stream.cuda_stream))
    assert st == lbibm.LB_OK
    torch.cuda.synchronize(dev)
    S, V = d_area.cpu().numpy(), d_vol.cpu().numpy()
    if empty_after is None:
        return S, V, None
    keep = np.ones(n_cells, bool)
    keep[empty_after + 1] = False
    return S[keep], V[keep], (S[empty_after + 1], V[empty_after + 1])


def test_noalloc_area_volume_matches_oracle_and_context_two_calls():
    import __graft_entry__
    import oracle

    __graft_entry__.build()
    meshes = _meshes()
    S0 = np.array([oracle.mesh_area_volume(m.rest, m.tris)[0] for m in meshes])
    V0 = np.array([oracle.mesh_area_volume(m.rest, m.tris)[1] for m in meshes])
    for call, (seed, amp) in enumerate([(1, 0.03), (2, 0.08)]):
        pos = _deformed(meshes, seed, amp)
        S, V, empty = _noalloc_area_volume(meshes, pos, empty_after=call)
        So = np.array([oracle.mesh_area_volume(x, m.tris)[0] for x, m in zip(pos, meshes)])
        Vo = np.array([oracle.mesh_area_volume(x, m.tris)[1] for x, m in zip(pos, meshes)])
        assert np.abs(S - So).max() <= 1e-10 * So.max(), (call, S, So)
        assert np.abs(V - Vo).max() <= 1e-10 * Vo.max(), (call, V, Vo)
        assert empty == (0.0, 0.0), (call, empty)
        Sc, Vc = _context_area_volume(meshes, pos)
        assert np.abs(S - Sc).max() <= (2e-8 * S0 + 1e-5 * np.abs(Sc - S0)).max(), (call, S, Sc)
        assert np.abs(V - Vc).max() <= (2e-8 * V0 + 1e-5 * np.abs(Vc - V0)).max(), (call, V, Vc)


def test_noalloc_no_cells_is_a_no_op():
    from paper_1110_0995_gb300 import lbibm

    L = lbibm.lib()
    starts = np.zeros(1, dtype=np.int32)
    st = L.ibm_area_volume_noalloc(None, None, None, starts.ctypes.data_as(ctypes.c_void_p), 0, None, None, None)
    assert st == lbibm.LB_OK


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
