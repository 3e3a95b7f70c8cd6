"""The C-ABI library loads and exports every entry point include/lbibm.h declares (no GPU needed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lbibm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:lb_status|const char\*|int)\s+(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("lb_create", "lb_set_obstacles", "ibm_add_mesh", "lb_step", "lb_get_fields", "lb_destroy"):
        assert required in names


def test_library_builds_and_exports_every_symbol():
    import __graft_entry__

    __graft_entry__.build()
    from paper_1110_0995_gb300 import lbibm

    L = lbibm.lib()
    for name in _declared():
        assert hasattr(L, name), name
    assert set(_declared()) == set(lbibm.EXPORTS)
    assert L.lb_version() >= 10000


def test_null_context_is_rejected_without_gpu():
    import ctypes
    from paper_1110_0995_gb300 import lbibm

    L = lbibm.lib()
    assert L.lb_step(None, 1) == lbibm.LB_ERR_ARG
    assert L.lb_destroy(None) == lbibm.LB_OK
    assert isinstance(L.lb_last_error(None), bytes)          # never NULL
    out = ctypes.c_void_p()
    p = lbibm.make_params((4, 4, 4), tau=0.5)
    assert L.lb_create(ctypes.byref(p), None, ctypes.byref(out)) == lbibm.LB_ERR_ARG
    assert not out.value
    assert b"tau must be > 1/2" in L.lb_last_error(None)


def test_binding_checks_caller_buffers():
    """The binding refuses a buffer the library would write past or read past
    (wrong dtype, layout, size) before any call crosses the C ABI."""
    import numpy as np

    from paper_1110_0995_gb300 import lbibm

    ok = np.zeros((10, 3))
    assert lbibm._f64_out(ok, 10) is ok
    assert lbibm._f64_out(np.zeros(40), 10) is not None          # larger is fine
    for bad in (np.zeros((9, 3)), np.zeros((10, 3), np.float32), np.zeros((3, 10)).T):
        with pytest.raises(ValueError):
            lbibm._f64_out(bad, 10)
    ro = np.zeros((10, 3))
    ro.flags.writeable = False
    with pytest.raises(ValueError):
        lbibm._f64_out(ro, 10)
    assert lbibm._f64_in(np.ones((10, 3), np.float32), 10).dtype == np.float64
    with pytest.raises(ValueError):
        lbibm._f64_in(np.ones((11, 3)), 10)
