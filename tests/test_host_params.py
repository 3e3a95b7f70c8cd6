"""lb_create / lb_create_batch refuse invalid lattice parameters on the host,
before any CUDA call (so this runs without a GPU)."""
import ctypes
import math

import pytest


@pytest.fixture(scope="module")
def lbibm():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1110_0995_gb300 import lbibm

    return lbibm


def _bad_params(lbibm):
    mk = lbibm.make_params
    yield "dims", mk((0, 8, 8))
    yield "too many nodes", mk((2048, 2048, 1024))
    yield "tau = 1/2", mk((8, 8, 8), tau=0.5)
    yield "tau nan", mk((8, 8, 8), tau=math.nan)
    yield "force inf", mk((8, 8, 8), body_force=(math.inf, 0.0, 0.0))
    yield "wall nan", mk((8, 8, 8), wall_velocity=((0, 0, 0), (math.nan, 0, 0)))
    yield "storage", mk((8, 8, 8), storage=7)
    p = mk((8, 8, 8))
    p.reserved[2] = 1
    yield "reserved", p


def test_invalid_params_are_refused_on_the_host(lbibm):
    L = lbibm.lib()
    for name, p in _bad_params(lbibm):
        h = ctypes.c_void_p(123)
        st = L.lb_create(ctypes.byref(p), None, ctypes.byref(h))
        assert st == lbibm.LB_ERR_ARG, name
        assert h.value is None, name          # *out is cleared
        arr = (lbibm.LbParams * 2)(lbibm.make_params((8, 8, 8)), p)
        assert L.lb_create_batch(arr, 2, None, ctypes.byref(h)) == lbibm.LB_ERR_ARG, name


def test_batch_arguments_are_refused_on_the_host(lbibm):
    L = lbibm.lib()
    h = ctypes.c_void_p()
    a, b = lbibm.make_params((8, 8, 8)), lbibm.make_params((8, 8, 8), storage="f16")
    mixed = (lbibm.LbParams * 2)(a, b)
    assert L.lb_create_batch(mixed, 2, None, ctypes.byref(h)) == lbibm.LB_ERR_ARG   # one storage per batch
    one = (lbibm.LbParams * 1)(a)
    assert L.lb_create_batch(one, 0, None, ctypes.byref(h)) == lbibm.LB_ERR_ARG
    assert L.lb_create_batch(one, 4097, None, ctypes.byref(h)) == lbibm.LB_ERR_ARG
    assert L.lb_create_batch(None, 1, None, ctypes.byref(h)) == lbibm.LB_ERR_ARG
    assert L.lb_create_batch(one, 1, None, None) == lbibm.LB_ERR_ARG


def test_bead_arguments_are_refused_on_the_host(lbibm):
    """bead_forces / bead_relax check their arguments before any CUDA call."""
    import numpy as np

    x = np.zeros((4, 3))
    x[:, 0] = np.arange(4) * 3.0
    m = np.tile([0.0, 0.0, 1.0], (4, 1))
    bad = [
        dict(xyz=x[:0], moments=m[:0], c=1.0, radius=1.0, k=1.0),                  # no beads
        dict(xyz=x, moments=m, c=1.0, radius=-1.0, k=1.0),                         # negative radius
        dict(xyz=x, moments=m, c=1.0, radius=1.0, k=-2.0),                         # negative stiffness
        dict(xyz=x, moments=m, c=math.nan, radius=1.0, k=1.0),                     # non-finite constant
        dict(xyz=x, moments=m, c=1.0, radius=1.0, k=1.0, box=(0.0, 1.0, 1.0), periodic=(1, 0, 0)),
    ]
    for kw in bad:
        with pytest.raises(lbibm.LbError) as e:
            lbibm.bead_forces(**kw)
        assert e.value.status == lbibm.LB_ERR_ARG
    with pytest.raises(lbibm.LbError) as e:
        lbibm.bead_relax(x, m, 1.0, 1.0, 1.0, 1.0, 0.1, steps=-1)
    assert e.value.status == lbibm.LB_ERR_ARG
    p = lbibm._bead_params(1.0, 1.0, 1.0)
    p.reserved[0] = 3
    L = lbibm.lib()
    F = np.zeros_like(x)
    assert L.bead_forces(lbibm._ptr(x), lbibm._ptr(m), 4, ctypes.byref(p), lbibm._ptr(F), None) == lbibm.LB_ERR_ARG


def test_context_free_calls_say_why(lbibm):
    """A failed call without a context leaves its reason for lb_last_error(NULL),
    per thread; the binding puts it into the exception."""
    import threading

    import numpy as np

    L = lbibm.lib()
    h = ctypes.c_void_p()
    p = lbibm.make_params((8, 8, 8), tau=0.4)
    assert L.lb_create(ctypes.byref(p), None, ctypes.byref(h)) == lbibm.LB_ERR_ARG
    assert "tau must be > 1/2" in lbibm.last_error()
    arr = (lbibm.LbParams * 2)(lbibm.make_params((8, 8, 8)), lbibm.make_params((8, 8, 8), storage="bf16"))
    assert L.lb_create_batch(arr, 2, None, ctypes.byref(h)) == lbibm.LB_ERR_ARG
    assert "same storage" in lbibm.last_error()
    with pytest.raises(lbibm.LbError, match="channel 1: wall velocities must be finite"):
        lbibm.Simulation([lbibm.make_params((8, 8, 8)),
                          lbibm.make_params((8, 8, 8), wall_velocity=((0, 0, 0), (0, math.inf, 0)))])
    with pytest.raises(lbibm.LbError, match="invalid bead parameters"):
        lbibm.bead_forces(np.zeros((2, 3)), np.zeros((2, 3)), 1.0, -1.0, 1.0)
    assert "invalid bead parameters" in lbibm.last_error()
    # another thread has its own message
    seen = []
    t = threading.Thread(target=lambda: seen.append(lbibm.last_error()))
    t.start()
    t.join()
    assert seen == ["no error"]
    x, tr = np.eye(3), np.array([[0, 1, 2]] * 4, np.int32)
    assert lbibm.check_mesh(x, tr) != ""
    assert ">= 4 nodes" in lbibm.last_error()


def test_batch_scenes_must_agree_on_context_settings(lbibm):
    """Collisions and point dynamics belong to the whole context: a batch of
    scenes that differ in them is refused before anything is created."""
    from paper_1110_0995_gb300 import scene

    a = scene.Scene(name="a", dims=(8, 8, 8))
    b = scene.Scene(name="b", dims=(8, 8, 8), ib_dynamics=(1.0, 0.5))
    c = scene.Scene(name="c", dims=(8, 8, 8), repulsion=(0.01, 1.0))
    for pair in ((a, b), (a, c)):
        with pytest.raises(ValueError, match="differ in"):
            lbibm.Simulation.from_scenes(list(pair))


def test_guard_zone_size_is_checked_on_the_host(lbibm):
    L = lbibm.lib()
    assert L.lb_set_guard_zones(1 << 31) == lbibm.LB_ERR_ARG
    assert "1 GiB" in lbibm.last_error()
    assert L.lb_set_guard_zones(4096) == lbibm.LB_OK
    assert L.lb_set_guard_zones(0) == lbibm.LB_OK


def test_fields_into_checks_its_buffers(lbibm):
    """The caller's field buffers must be contiguous float32 arrays of N and
    3 N values; anything else is refused in the binding, before the C ABI is
    called (no context is needed to see it)."""
    import numpy as np

    sim = lbibm.Simulation.__new__(lbibm.Simulation)
    sim.dims = [(4, 4, 4)]
    sim.channel = 0
    rho, u = np.empty(64, np.float32), np.empty(192, np.float32)
    bad = [(np.empty(64, np.float64), u), (rho, np.empty(191, np.float32)),
           (np.empty(128, np.float32)[::2], u), (rho, np.empty((3, 64), np.float32).T)]
    for r, v in bad:
        with pytest.raises(ValueError, match="contiguous float32"):
            sim.fields_into(r, v)
