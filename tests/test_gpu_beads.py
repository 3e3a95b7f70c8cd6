"""Magnetic bead assembly on the GPU (through the C ABI) against the FP64
oracle: dipole + contact forces of all pairs (FP32 on the device) and the
overdamped bead motion.

Inputs are rounded to FP32 first (the device stores FP32 positions and
moments; at |x| ~ 40 a position carries ~2e-6 lu, which the 1/r^4 force of a
close pair would amplify) and no two beads start closer than 1.2 R.
Tolerances: forces within 1e-5 of the largest force magnitude (FP32 sums of
a few hundred terms); positions within 2e-5 lu after short runs.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def _beads(n, seed, L=40.0, R=1.0):
    rng = np.random.default_rng(seed)
    pts = []
    while len(pts) < n:   # no two beads closer than 1.2 R (minimum image)
        p = rng.uniform(0.0, L, size=3)
        if pts:
            d = np.asarray(pts) - p
            d -= L * np.round(d / L)
            if (d * d).sum(axis=1).min() < (1.2 * R) ** 2:
                continue
        pts.append(p)
    x = np.asarray(pts, np.float32).astype(np.float64)
    m = (np.tile([0.0, 0.0, 1.0], (n, 1)) + 0.2 * rng.normal(size=(n, 3))).astype(np.float32).astype(np.float64)
    return x, m


@pytest.mark.parametrize("n,periodic", [(1, (0, 0, 0)), (300, (1, 1, 1)), (513, (0, 0, 1)), (256, (0, 0, 0))])
def test_forces_match_oracle(n, periodic):
    from paper_1110_0995_gb300 import lbibm

    x, m = _beads(n, seed=n)
    box = (40.0, 40.0, 40.0)
    F = lbibm.bead_forces(x, m, 2.0, 1.0, 5.0, box, periodic)
    Fo = oracle.bead_forces(x, m, 2.0, 1.0, 5.0, box, periodic)
    if n == 1:
        assert np.all(F == 0.0)
        return
    assert np.abs(F - Fo).max() <= 1e-5 * np.abs(Fo).max()


def test_pair_relaxes_to_force_balance():
    from paper_1110_0995_gb300 import lbibm

    x0 = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 3.0]])
    m = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 1.0]])
    x = lbibm.bead_relax(x0, m, 1.0, 1.0, 10.0, mobility=1.0, dt=0.02, steps=3000)
    xo = oracle.bead_relax(x0, m, 1.0, 1.0, 10.0, mobility=1.0, dt=0.02, steps=3000)
    assert np.abs(x - xo).max() < 1e-5


def test_short_assembly_matches_oracle():
    from paper_1110_0995_gb300 import lbibm

    x, m = _beads(200, seed=3, L=24.0)
    box = (24.0, 24.0, 24.0)
    args = dict(c=0.5, radius=1.0, k=5.0, mobility=0.2, dt=0.05, steps=20, box=box, periodic=(1, 1, 1))
    xg = lbibm.bead_relax(x, m, **args)
    xo = oracle.bead_relax(x, m, **args)
    d = xg - xo
    d -= 24.0 * np.round(d / 24.0)   # a bead may wrap on one side and not the other
    assert np.abs(d).max() < 2e-5
    assert np.abs(xo - x).max() > 1e-3   # the beads did move


def test_bad_arguments():
    from paper_1110_0995_gb300 import lbibm

    x, m = _beads(4, seed=1)
    with pytest.raises(lbibm.LbError):
        lbibm.bead_forces(x[:0], m[:0], 1.0, 1.0, 1.0)
    with pytest.raises(lbibm.LbError):
        lbibm.bead_forces(x, m, 1.0, -1.0, 1.0)
    with pytest.raises(lbibm.LbError):
        lbibm.bead_relax(x, m, 1.0, 1.0, 1.0, 1.0, 0.1, steps=3, box=(0.0, 1.0, 1.0), periodic=(1, 0, 0))
