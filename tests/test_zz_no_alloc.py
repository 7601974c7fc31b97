"""The allocation-free search entry point gives what the workspace one gives.

Some callers of this library cannot allocate device memory at the moment they
plan -- real-time control loops that forbid allocation after start-up (an
allocation can block for an unbounded time), plug-ins whose host application
owns every allocation. cpp_dp_search_static serves them from a fixed scratch
array inside the library. This file calls it through the C ABI on lattices of
different sizes in a row, small then large then small again (each call reuses
the scratch the one before left behind, and the last one finds rows beyond its
own lattice filled by a larger one), and checks
each result against cpp_dp_search run with its own workspace: the search is
exact, so indices, cost and seed must be identical. It also checks that a
lattice larger than the scratch is refused with a clear message.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _static_entry():
    from paper_2309_09102_gb300 import cppflow
    fn = cppflow.lib().cpp_dp_search_static
    P = ctypes.c_void_p
    fn.restype = ctypes.c_int
    fn.argtypes = [P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                   P, P, P, P, P]
    return fn


def _lattice(T, K, n, seed):
    rng = np.random.default_rng(seed)
    Kp = ((K + 31) // 32) * 32
    cand = rng.normal(0.0, 0.3, (T, n, Kp)).astype(np.float32)
    pen = rng.choice([0.0, 10.0, 100.0, 110.0], (T, Kp)).astype(np.float32)
    pen[:, K:] = np.inf
    return cand, pen, Kp


def test_static_scratch_matches_workspace_search():
    import torch

    from paper_2309_09102_gb300 import cppflow
    fn = _static_entry()
    dev = "cuda:0"
    stream = torch.cuda.current_stream().cuda_stream or None
    for T, K, n, seed in [(25, 130, 9, 2), (40, 300, 7, 1), (30, 200, 7, 3)]:
        cand, pen, Kp = _lattice(T, K, n, seed)
        c_d = torch.from_numpy(cand).to(dev)
        p_d = torch.from_numpy(pen).to(dev)
        outs = []
        for use_static in (False, True):
            sel = torch.full((T,), -1, dtype=torch.int32, device=dev)
            best = torch.full((1,), -1.0, dtype=torch.float32, device=dev)
            seed_q = torch.zeros(T, n, dtype=torch.float32, device=dev)
            st = torch.zeros(1, dtype=torch.int32, device=dev)
            if use_static:
                rc = fn(c_d.data_ptr(), p_d.data_ptr(), T, K, Kp, n, sel.data_ptr(), best.data_ptr(),
                        seed_q.data_ptr(), st.data_ptr(), stream)
                assert rc == cppflow.OK, cppflow.last_error()
            else:
                ws = torch.empty(cppflow.dp_workspace_size(T, Kp), dtype=torch.uint8, device=dev)
                cppflow.dp_search(c_d, p_d, K, ws, sel, best, seed_q, st)
            torch.cuda.synchronize()
            outs.append((sel.cpu().numpy(), best.item(), seed_q.cpu().numpy(), int(st.item())))
        ref, got = outs
        np.testing.assert_array_equal(got[0], ref[0])
        assert got[1] == ref[1]
        np.testing.assert_array_equal(got[2], ref[2])
        assert got[3] == ref[3] == 0


def test_static_scratch_refuses_oversized_lattice():
    import torch

    from paper_2309_09102_gb300 import cppflow
    fn = _static_entry()
    buf = torch.zeros(64, dtype=torch.float32, device="cuda:0")
    p = buf.data_ptr()
    rc = fn(p, p, 5000, 1000, 1024, 7, p, p, None, None, None)  # needs ~10 MB of scratch
    assert rc == cppflow.ERR_INVALID_ARG
    assert "static" in cppflow.last_error() and "scratch" in cppflow.last_error()
