"""The C-ABI library loads and exports every function that include/*.h declares
(no GPU needed: nothing is called that would touch a device)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(cpp_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2309_09102_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("cpp_fk_batch", "cpp_mask", "cpp_dp_search", "cpp_lm_refine", "cpp_check",
                     "cpp_plan", "cpp_plan_batch", "cpp_dp_workspace_size", "cpp_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls(lib):
    from paper_2309_09102_gb300 import cppflow
    p = cppflow.make_params()
    assert p.lm_iters == 20 and abs(p.tau_pos - 1e-3) < 1e-18
    assert cppflow.lib().cpp_version() >= 100
    assert cppflow.dp_workspace_size(300, 512) >= 300 * 512 * 2
    # host-side validation rejects bad arguments before touching a device
    r = cppflow.make_robot([0.1] * 7, [0.1] * 7, [0.0] * 7, [-1] * 7, [1] * 7)
    st = cppflow.lib().cpp_mask(ctypes.byref(r), ctypes.byref(p), None, None, 0, 1, 4,
                                None, None, None, None, None)
    assert st == cppflow.ERR_INVALID_ARG
    assert "T" in cppflow.last_error()
    bad = cppflow.make_robot([0.1] * 7, [0.1] * 7, [0.0] * 7, [1] * 7, [-1] * 7)
    assert cppflow.lib().cpp_check(ctypes.byref(bad), ctypes.byref(p), None, None, 5, None, None,
                                   None) == cppflow.ERR_INVALID_ARG


def test_diagnostics_and_batch_knobs_are_validated_on_the_host(lib):
    """Bad arguments of the bounded-wait self-test and of the batch schedule knobs are
    refused before any device work."""
    from paper_2309_09102_gb300 import cppflow
    L = cppflow.lib()
    dummy = ctypes.c_void_p(8)  # never dereferenced: the limit is checked first
    assert L.cpp_wait_selftest(10, 0, dummy, None) == cppflow.ERR_INVALID_ARG
    assert "limit" in cppflow.last_error()
    assert L.cpp_wait_selftest(2 * 10 ** 10, 1, dummy, None) == cppflow.ERR_INVALID_ARG
    assert L.cpp_wait_selftest(10 ** 6, 0, None, None) == cppflow.ERR_INVALID_ARG
    assert L.cpp_batch_set_mask_tasks(None, 4) == cppflow.ERR_INVALID_ARG
    assert L.cpp_batch_set_cluster_min_kp(None, 512, None) == cppflow.ERR_INVALID_ARG
    assert L.cpp_batch_set_split(None, 1.0, 64, None) == cppflow.ERR_INVALID_ARG


def test_smoothing_params_are_validated_on_the_host(lib):
    """smooth_lambda must be positive, smooth_rounds within [0, 1000], and the
    trajectory-length step's (n + 1) T doubles must fit in shared memory; every
    check fails before any device pointer is touched."""
    from paper_2309_09102_gb300 import cppflow
    L = cppflow.lib()
    r = cppflow.make_robot([0.1] * 7, [0.1] * 7, [0.0] * 7, [-1] * 7, [1] * 7)
    p = cppflow.make_params()
    assert p.smooth_rounds == 0 and p.smooth_lambda == 1.0
    fake = ctypes.c_void_p(256)  # never dereferenced: validation fails first
    for kw in ({"smooth_lambda": 0.0}, {"smooth_lambda": float("nan")}, {"smooth_rounds": -1},
               {"smooth_rounds": 1001}):
        q = cppflow.make_params(**kw)
        assert L.cpp_lm_refine(ctypes.byref(r), ctypes.byref(q), fake, fake, 10, fake, None, None,
                               None) == cppflow.ERR_INVALID_ARG
    big = cppflow.make_params(smooth_rounds=1)
    assert L.cpp_lm_refine(ctypes.byref(r), ctypes.byref(big), fake, fake, 4000, fake, None, None,
                           None) == cppflow.ERR_INVALID_ARG
    assert "227" in cppflow.last_error()
    assert L.cpp_smooth_step(ctypes.byref(r), ctypes.byref(p), fake, fake, 4000, None,
                             None) == cppflow.ERR_INVALID_ARG


def test_collision_models_are_validated_on_the_host(lib):
    """A capsule paired with itself, a frame above n, too many boxes or a negative
    radius: INVALID_ARG before any device pointer is touched."""
    import numpy as np
    from paper_2309_09102_gb300 import cppflow, synth
    L = cppflow.lib()
    arm = synth.draw_arm(2, 7)
    r = cppflow.robot_from_arm(arm)
    p = cppflow.make_params()
    assert p.pen_collide == 100.0
    fake = ctypes.c_void_p(256)
    good = cppflow.geometry_from(synth.with_boxes(synth.link_capsules(arm), 1, 2))

    def call(g):
        return L.cpp_mask_geo(ctypes.byref(r), ctypes.byref(p), ctypes.byref(g), fake, fake, 4, 8, 8,
                              fake, fake, None, None, None, None)

    for tweak in ("self_pair", "frame", "boxes", "radius"):
        g = cppflow.geometry_from(synth.with_boxes(synth.link_capsules(arm), 1, 2))
        if tweak == "self_pair":
            g.pairs[0][1] = g.pairs[0][0]
        elif tweak == "frame":
            g.caps[0].frame = 8
        elif tweak == "boxes":
            g.n_boxes = 9
        else:
            g.caps[1].radius = -0.01
        assert call(g) == cppflow.ERR_INVALID_ARG, tweak
        assert "collision model" in cppflow.last_error()
    bad_p = cppflow.make_params(pen_collide=float("inf"))
    assert L.cpp_mask_geo(ctypes.byref(r), ctypes.byref(bad_p), ctypes.byref(good), fake, fake, 4, 8,
                          8, fake, fake, None, None, None, None) == cppflow.ERR_INVALID_ARG
    assert good.n_caps == 7 and good.n_pairs == 15 and good.n_boxes == 2
    assert np.isclose(good.caps[0].radius, 0.03)
