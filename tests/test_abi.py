"""The C-ABI library loads and exports every function include/mppi.h declares
(no GPU needed: nothing here launches a kernel)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(mppi_[a-z0-9_]+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    import paper_2409_07563_gb300 as m
    m.build()
    from paper_2409_07563_gb300 import _lib
    return _lib.load()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("mppi_create", "mppi_step", "mppi_destroy", "mppi_step_backward",
                     "mppi_set_stream", "mppi_poll_status", "mppi_sample_noise"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_library_rejects_bad_arguments_without_a_gpu(lib):
    import ctypes
    from paper_2409_07563_gb300 import _lib
    h = ctypes.c_void_p()
    # NULL descriptors are rejected on the host, before any CUDA call
    assert lib.mppi_create(None, None, 16, 8, 0.01, 1.0, None, None, ctypes.byref(h)) == 1
    assert h.value is None
    assert lib.mppi_step(None, None, None, None, None, None, None) == 1
    assert lib.mppi_sample_noise(0, 0, -1, 4, None, None, None) == 1
    opt = _lib.Options()
    lib.mppi_default_options(ctypes.byref(opt))
    assert opt.beta == 1 and opt.precision == 0 and opt.seed == 0


def test_checked_option_is_validated_on_the_host(lib):
    """mppi_options.checked takes 0 or 1; anything else is rejected before
    any CUDA call (so this runs without a GPU)."""
    import ctypes
    import numpy as np
    from paper_2409_07563_gb300 import _lib
    import workloads as W
    p = W.cartpole(K=16, T=8)
    dyn_p = np.asarray(p["dyn_params"], np.float32)
    cost_p = np.asarray(p["cost_params"], np.float32)
    sig = np.asarray(p["sigma"], np.float32)
    fp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    dyn = _lib.DynamicsDesc(p["dyn_kind"], p["integrator"], 4, 1, fp(dyn_p), dyn_p.size)
    cost = _lib.CostDesc(p["cost_kind"], fp(cost_p), cost_p.size, None, 0, 0)
    opt = _lib.Options()
    lib.mppi_default_options(ctypes.byref(opt))
    assert opt.checked == 0 and list(opt.reserved) == [0] * 5
    h = ctypes.c_void_p()
    for bad in (2, -1):
        opt.checked = bad
        st = lib.mppi_create(ctypes.byref(dyn), ctypes.byref(cost), 16, 8, 0.02, 1.0, fp(sig),
                             ctypes.byref(opt), ctypes.byref(h))
        assert st == 1 and h.value is None
    # the struct layout: checked follows rollout_variant, then five reserved ints
    assert _lib.Options.checked.offset == _lib.Options.rollout_variant.offset + 4
    assert ctypes.sizeof(_lib.Options) == _lib.Options.reserved.offset + 5 * 4
