"""The library's mesh check (`ibm_check_mesh`, the host code `ibm_add_mesh`
runs before it accepts a cell membrane) on the CPU: the cell meshes of the
workloads pass, and each kind of broken mesh is refused with its reason."""
import numpy as np
import pytest

from paper_1110_0995_gb300 import scene


@pytest.fixture(scope="module")
def lbibm():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1110_0995_gb300 import lbibm

    return lbibm


def _outward(x, t):
    a, b, c = x[t[:, 0]], x[t[:, 1]], x[t[:, 2]]
    vol = np.einsum("ij,ij->", a, np.cross(b, c)) / 6.0
    return t if vol > 0 else t[:, ::-1].copy()


def _bipyramid(m):
    """Two apexes over an m-gon: the apexes have valence m."""
    ang = 2 * np.pi * np.arange(m) / m
    x = np.vstack([np.column_stack([np.cos(ang), np.sin(ang), np.zeros(m)]), [[0, 0, 1.0]], [[0, 0, -1.0]]])
    top, bot = m, m + 1
    t = [(top, k, (k + 1) % m) for k in range(m)] + [(bot, (k + 1) % m, k) for k in range(m)]
    return x, _outward(x, np.array(t, np.int32))


@pytest.mark.parametrize("kind", ["rbc", "ctc", "ico0", "ico3", "t1rbc", "t1ctc", "bipyramid64"])
def test_cell_meshes_pass(lbibm, kind):
    if kind in ("rbc", "ctc"):
        x, t = scene.cell_template(kind)
    elif kind.startswith("ico"):
        x, t = scene.icosphere(int(kind[3:]))
    elif kind.startswith("t1"):
        pytest.importorskip("scipy")
        x, t = scene.table1_template(kind[2:])
    else:
        x, t = _bipyramid(64)
    assert lbibm.check_mesh(x + 10.0, t) == ""


def test_broken_meshes_are_refused(lbibm):
    x, t = scene.icosphere(1)
    n = len(x)
    cases = {
        "open": (x, t[1:], "not closed"),
        "inward": (x, t[:, ::-1], "volume must be positive"),
        "face twice": (x, np.concatenate([t, t[:1]]), "edge used twice"),
        "index high": (x, np.where(np.arange(t.size).reshape(t.shape) == 0, n, t), "out of range"),
        "index negative": (x, np.where(np.arange(t.size).reshape(t.shape) == 4, -1, t), "out of range"),
        "isolated node": (np.vstack([x, [[0.0, 0.0, 0.0]]]), t, "isolated node"),
        "too small": (x[:3], np.array([[0, 1, 2]] * 4, np.int32), ">= 4 nodes"),
        "not finite": (np.where(np.arange(x.size).reshape(x.shape) == 5, np.nan, x), t, "finite"),
        "too far": (x + 5.0e6, t, "|x| < 4e6"),
        "valence 65": (*_bipyramid(65), "valence > 64"),
    }
    deg = t.copy()
    deg[0, 1] = deg[0, 0]
    cases["degenerate"] = (x, deg, "degenerate")
    # two tetrahedra sharing one vertex: closed and outward, but that vertex is two fans
    xt, tt = scene.icosphere(0)
    tet_x = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1.0]])
    tet_t = _outward(tet_x, np.array([[0, 2, 1], [0, 1, 3], [0, 3, 2], [1, 2, 3]], np.int32))
    bow_x = np.vstack([tet_x, -tet_x[1:]])
    bow_t = np.vstack([tet_t, np.where(tet_t == 0, 0, tet_t + 3)])
    bow_t[4:] = _outward(bow_x, bow_t[4:])
    cases["bowtie"] = (bow_x, bow_t, "single fan")
    for name, (xx, tt, reason) in cases.items():
        why = lbibm.check_mesh(xx, tt)
        assert reason in why, (name, why)


def test_random_corruptions_agree_with_a_direct_edge_count(lbibm):
    """Drop, duplicate or flip random faces of an icosphere; the library
    accepts exactly the meshes in which every directed edge appears once and
    its reverse once (all others here have a bad edge)."""
    rng = np.random.default_rng(7)
    x, t = scene.icosphere(2)
    for _ in range(40):
        tt = t.copy()
        op = rng.integers(3)
        k = rng.integers(len(tt))
        if op == 0:
            tt = np.delete(tt, k, axis=0)
        elif op == 1:
            tt = np.concatenate([tt, tt[k:k + 1]])
        else:
            tt[k] = tt[k, ::-1]
        e = np.concatenate([tt[:, [0, 1]], tt[:, [1, 2]], tt[:, [2, 0]]])
        keys = {tuple(r) for r in e}
        ok = len(keys) == len(e) and all((b, a) in keys for a, b in keys)
        assert (lbibm.check_mesh(x, tt) == "") == ok
        assert not ok
