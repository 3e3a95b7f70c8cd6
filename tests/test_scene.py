"""Seeded synthetic inputs: determinism and the sizes the workloads state."""
import numpy as np

from paper_1110_0995_gb300 import scene


def test_plain_channel_is_deterministic_and_sized():
    a, b = scene.channel_plain(seed=3), scene.channel_plain(seed=3)
    assert a.dims == (32, 16, 64) and a.n_ib_nodes == 642 and a.meshes[0].n_tris == 1280
    assert np.array_equal(a.meshes[0].rest, b.meshes[0].rest)
    assert not np.array_equal(a.meshes[0].rest, scene.channel_plain(seed=4).meshes[0].rest)


def test_positions_are_quantized_and_clear_of_walls():
    sc = scene.micropost_filter()
    assert len(sc.spheres) == 120 and len(sc.meshes) == 62 and sc.n_ib_nodes == 43644
    for m in sc.meshes:
        q = m.rest / scene.POS_QUANTUM
        assert np.array_equal(q, np.round(q))
        for ax in (1, 2):
            assert m.rest[:, ax].min() >= -0.5 + scene.WALL_CLEARANCE
            assert m.rest[:, ax].max() <= sc.dims[ax] - 0.5 - scene.WALL_CLEARANCE
    s = sc.spheres.astype(np.float64) / scene.SPHERE_QUANTUM
    assert np.array_equal(s, np.round(s))


def test_large_filter_counts():
    sc = scene.micropost_filter_large()
    assert sc.dims == (512, 256, 128) and len(sc.spheres) == 672
    assert sc.n_ib_nodes == 400 * 642 + 4 * 2562


def test_gap_sweep_channels():
    ch = scene.gap_sweep()
    assert len(ch) == 24
    for c in ch:
        nx, ny, nz = c.dims
        assert 64 <= nx <= 256 and 32 <= ny <= 128 and 32 <= nz <= 64
        assert nx % 8 == 0 and ny % 8 == 0 and nz % 8 == 0
        assert 1 <= len(c.meshes) <= 40
