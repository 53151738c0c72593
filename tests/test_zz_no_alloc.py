"""nlos_solve_static: the FFT solve for callers that cannot allocate device
memory while they solve (e.g. inside a CUDA-graph stream capture, under a
fixed memory budget or another framework's allocator).  Its scratch is a
static device array, so this test checks, through the C ABI, that two calls
in a row agree with the plan-based nlos_solve, and that grids beyond the
static maximum are refused.  It sits in its own file, collected last."""

import ctypes

import numpy as np
import pytest

from tests.gpu_util import dev, host, rel_l2

pytestmark = pytest.mark.gpu


def _static_solve(lib, n, nt, rhs_t, x_t, c0, c1):
    import torch
    return lib.nlos_solve_static(n, n, nt, ctypes.c_void_p(rhs_t.data_ptr()), ctypes.c_void_p(x_t.data_ptr()),
                                 c0, c1, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_solve_static_matches_nlos_solve_twice_in_a_row():
    import torch
    from paper_2301_00406_gb300 import nlos
    lib = nlos.load()
    cases = [(32, 256, 93.4, 0.1, 1), (64, 512, 3.0, 800.0, 2)]
    for n, nt, c0, c1, seed in cases:
        rhs = dev(np.random.default_rng(seed).standard_normal((n, n, nt)))
        x_static = torch.full_like(rhs, float("nan"))
        assert _static_solve(lib, n, nt, rhs, x_static, c0, c1) == 0, nlos.last_error()
        plan = nlos.Plan(n, n, nt, 16e-12)
        x_plan = nlos.solve_t(plan, rhs, c0, c1)
        assert rel_l2(host(x_static), host(x_plan)) < 1e-5
        plan.close()


def test_solve_static_rejects_grids_beyond_its_scratch():
    import torch
    from paper_2301_00406_gb300 import nlos
    lib = nlos.load()
    buf = torch.zeros(8, device="cuda")
    for n, nt in [(128, 64), (64, 1024), (48, 64), (32, 8)]:
        assert _static_solve(lib, n, nt, buf, buf, 1.0, 1.0) == -1
    assert "static" in nlos.last_error() or "powers of two" in nlos.last_error()
