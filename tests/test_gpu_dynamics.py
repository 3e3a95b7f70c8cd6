"""IB points with mass on the GPU (through the C ABI) against the FP64 oracle:
kick by the membrane + collision forces, exact drag drift with the fluid
velocity of the last collision, the drag impulse spread to the fluid.

Tolerances as for the massless path: velocity field relative L2 <= 1e-5 and
node positions <= 1e-5 lu; point velocities within 1e-4 of their largest
magnitude (FP32 sums of a few hundred kicks and drifts: measured 2e-5).
"""
import numpy as np
import pytest

import oracle
from paper_1110_0995_gb300 import scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


def _sim(*a, **k):
    from paper_1110_0995_gb300 import lbibm

    return lbibm.Simulation.from_scene(*a, **k)


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, float) - b) / np.linalg.norm(b))


def _compare(sc, steps):
    sim = _sim(sc)
    ref = oracle.System.from_scene(sc)
    sim.step(steps)
    ref.step(steps)
    _, u = sim.fields()
    _, uo = ref.fields()
    assert rel_l2(u, uo) < 1e-5
    for m in range(len(sc.meshes)):
        assert np.abs(sim.nodes(m) - ref.nodes(m)).max() < 1e-5
        vo = ref.velocities(m)
        assert np.abs(sim.velocities(m) - vo).max() <= 1e-4 * np.abs(vo).max()
    return sim, ref


# (light and overdamped; heavy and weakly coupled).  The exchange with the
# fluid is explicit: a light point with weak drag (m = 0.1, gamma = 0.1) blows
# up, and m = 0.05, gamma = 1 has a local burst near step 70 (the oracle as
# well), where FP32 and FP64 part ways; these two track the massless flow.
@pytest.mark.parametrize("m,gamma", [(0.05, 5.0), (2.0, 0.05)])
def test_small_filter_with_massive_points(m, gamma):
    """96x48x32 filter, posts, 4 red cells and a tumor cell, 200 cycles."""
    sc = scene.small_filter(seed=5, steps=200)
    sc.ib_dynamics = (m, gamma)
    sim, ref = _compare(sc, sc.steps)
    assert np.abs(ref.velocities(0)).max() > 1e-5   # the points do move on their own


def test_plain_channel_1000_steps_with_massive_points():
    sc = scene.channel_plain(seed=1, steps=1000)
    sc.ib_dynamics = (0.05, 5.0)
    _compare(sc, sc.steps)


def test_momentum_exchange_balances():
    """Periodic box, no walls or obstacles: the fluid's momentum (sum of the
    stored populations times e) gains what the points' m * W lose."""
    x, t = scene.icosphere(2)
    rng = np.random.default_rng(7)
    rest = 3.0 * x + np.array([12.2, 10.1, 9.8])
    xd = scene.quantize(rest + 0.1 * rng.standard_normal(rest.shape), scene.POS_QUANTUM)
    sc = scene.Scene(name="box", dims=(24, 20, 20), tau=0.9, body_force=(0, 0, 0), periodic=(1, 1, 1),
                     meshes=[scene.Mesh("rbc", rest, t, (0.02, 0.01, 0.01, 0.5, 0.9))], steps=0,
                     ib_dynamics=(0.7, 0.4))
    sim = _sim(sc)
    sim.set_nodes(0, xd)
    e, _, _ = oracle.constants()
    mass = 0.7

    def momentum():
        f = sim.populations().astype(np.float64)
        return (e.T.astype(float) @ f).sum(axis=1) + mass * sim.velocities(0).sum(axis=0)

    p0 = momentum()
    exch = 0.0
    for _ in range(10):
        sim.step(5)
        exch = max(exch, mass * np.abs(sim.velocities(0)).sum())
        assert np.abs(momentum() - p0).max() <= 1e-4 * exch
    assert exch > 1e-4


def test_dynamics_arguments_and_state():
    from paper_1110_0995_gb300 import lbibm

    sc = scene.channel_plain(seed=1, steps=0)
    sim = _sim(sc)
    for bad in ((-1.0, 1.0), (1.0, -0.5), (float("nan"), 1.0)):
        with pytest.raises(lbibm.LbError):
            sim.set_ib_dynamics(*bad)
    sim.set_ib_dynamics(1.0, 1.0)
    assert np.all(sim.velocities(0) == 0.0)
    sim.step(3)
    with pytest.raises(lbibm.LbError):
        sim.set_ib_dynamics(0.5, 1.0)   # only before the first step


def test_checkpoint_resume_with_massive_points():
    """A checkpoint of a context whose points carry mass holds their
    velocities: resuming from it repeats the same 60 cycles, and a massless
    context refuses it."""
    sc = scene.small_filter(seed=5, steps=0)
    sc.ib_dynamics = (2.0, 0.05)
    sim = _sim(sc)
    sim.step(80)
    state = sim.save_state()
    sim.step(60)
    xa, va, (_, ua) = sim.nodes(0), sim.velocities(0), sim.fields()
    assert np.abs(va).max() > 1e-6
    sim.step(40)                       # move the velocities away from the saved ones
    sim.load_state(state)
    assert sim.steps_done == 80
    sim.step(60)
    xb, vb, (_, ub) = sim.nodes(0), sim.velocities(0), sim.fields()
    assert np.abs(xa - xb).max() < 1e-7
    assert np.abs(va - vb).max() <= 1e-5 * np.abs(va).max()
    assert rel_l2(ub, ua) < 1e-6
    from paper_1110_0995_gb300 import lbibm

    sc.ib_dynamics = None
    plain = _sim(sc)
    with pytest.raises(lbibm.LbError):
        plain.load_state(state)
