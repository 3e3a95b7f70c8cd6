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


def _min_image(d, dims, periodic):
    d = d.copy()
    for ax in range(3):
        if periodic[ax]:
            d[..., ax] -= dims[ax] * np.round(d[..., ax] / dims[ax])
    return d


def test_filter_cells_clear_of_beads_and_each_other():
    """The recipe's placement: every node >= 1.5 lu from every bead surface
    (minimum image along the periodic axis), cell bounding spheres 1 lu apart."""
    sc = scene.micropost_filter()
    sph = sc.spheres.astype(np.float64)
    centres, radii = [], []
    for m in sc.meshes:
        d = _min_image(m.rest[:, None, :] - sph[None, :, :3], sc.dims, sc.periodic)
        gap = np.linalg.norm(d, axis=2) - sph[None, :, 3]
        assert gap.min() >= scene.WALL_CLEARANCE - 1e-2
        c = m.rest.mean(axis=0)
        centres.append(c)
        radii.append(np.linalg.norm(m.rest - c, axis=1).max())
    for i in range(len(centres)):
        for j in range(i):
            d = _min_image(centres[i] - centres[j], sc.dims, sc.periodic)
            # centroids stand in for the placement centres (a red cell's
            # biconcave profile is symmetric, so they agree to round-off)
            assert np.linalg.norm(d) >= radii[i] + radii[j] + 1.0 - 1e-6


def test_posts_are_chains_of_touching_beads():
    sc = scene.micropost_filter()
    s = sc.spheres.astype(np.float64)
    assert np.allclose(s[:, 3], scene.BEAD_RADIUS)
    for key in {(x, y) for x, y in s[:, :2]}:
        z = np.sort(s[(s[:, 0] == key[0]) & (s[:, 1] == key[1]), 2])
        assert len(z) == 10
        assert np.allclose(z, 2.5 + 2 * scene.BEAD_RADIUS * np.arange(10), atol=1e-2)


def test_workload_meshes_pass_the_library_check():
    """Every cell mesh of the workloads is one that ibm_add_mesh accepts (the
    library's host-side check; no GPU)."""
    import __graft_entry__

    __graft_entry__.build()
    from paper_1110_0995_gb300 import lbibm

    seen = set()
    for sc in (scene.channel_plain(seed=3), scene.micropost_filter(), scene.small_filter()):
        for m in sc.meshes:
            assert lbibm.check_mesh(m.rest, m.tris) == "", (sc.name, m.kind)
            seen.add(m.kind)
    assert seen == {"rbc", "ctc"}
