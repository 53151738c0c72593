"""nlos_solve_static: the FFT solve for callers that cannot allocate device
memory while they solve (code whose device memory belongs to another
allocator or to a fixed budget, real-time loops that must stay off the
driver's allocation path).  Its scratch is a static device array, so these
tests check, through the C ABI:

* results against the FP64 oracle's FFT solve element by element, at every
  lateral size (8-64) and at short and long time axes, and against the
  plan-based nlos_solve, with two calls in a row on the same grid (the
  second call reuses the scratch the first one left behind);
* in-place use (rhs and x the same buffer);
* that a call at an already-seen size leaves the device's free memory
  unchanged;
* that a fresh process whose very first call runs on a stream that does not
  wait for the legacy default stream gets the right answer (the set-up's
  table copies are finished before it returns);
* that grids beyond the static maximum are refused.

It sits in its own file, collected last."""

import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import admm
from tests.gpu_util import dev, host, rel_l2

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CASES = [(8, 16, 2.0, 0.7), (16, 64, 93.4, 0.1), (32, 256, 5.0, 3.0), (64, 512, 3.0, 800.0), (64, 16, 1.5, 2.0)]


def _static_solve(lib, n, nt, rhs_t, x_t, c0, c1, stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return lib.nlos_solve_static(n, n, nt, ctypes.c_void_p(rhs_t.data_ptr()), ctypes.c_void_p(x_t.data_ptr()),
                                 c0, c1, ctypes.c_void_p(s.cuda_stream))


def _check_against_oracle(x, rhs_np, c0, c1):
    want = admm.fft_solve(rhs_np, c0, c1)
    err = rel_l2(x, want)
    worst = float(np.max(np.abs(x - want))) / float(np.max(np.abs(want)))
    assert err < 1e-5 and worst < 1e-5, (err, worst)
    return err


@pytest.mark.parametrize("n,nt,c0,c1", CASES)
def test_solve_static_against_oracle_twice_in_a_row(n, nt, c0, c1):
    import torch
    from paper_2301_00406_gb300 import nlos
    lib = nlos.load()
    plan = nlos.Plan(n, n, nt, 16e-12)
    for call in range(2):                      # same grid, two calls in a row, different data
        rhs_np = np.random.default_rng(100 * n + nt + call).standard_normal((n, n, nt))
        rhs = dev(rhs_np)
        x_static = torch.full_like(rhs, float("nan"))
        assert _static_solve(lib, n, nt, rhs, x_static, c0, c1) == 0, nlos.last_error()
        x = host(x_static).astype(np.float64)
        err = _check_against_oracle(x, rhs_np, c0, c1)
        x_plan = host(nlos.solve_t(plan, rhs, c0, c1)).astype(np.float64)
        assert rel_l2(x, x_plan) < 1e-5
        print(f"n {n} nt {nt} call {call}: rel L2 vs oracle {err:.2e}")
    plan.close()


def test_solve_static_in_place_and_no_allocation():
    import torch
    from paper_2301_00406_gb300 import nlos
    lib = nlos.load()
    n, nt, c0, c1 = 32, 128, 4.0, 1.5
    rhs_np = np.random.default_rng(7).standard_normal((n, n, nt))
    buf = dev(rhs_np)
    assert _static_solve(lib, n, nt, buf, buf, c0, c1) == 0, nlos.last_error()   # size seen, set-up done
    torch.cuda.synchronize()
    _check_against_oracle(host(buf).astype(np.float64), rhs_np, c0, c1)
    buf.copy_(dev(rhs_np))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert _static_solve(lib, n, nt, buf, buf, c0, c1) == 0, nlos.last_error()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    _check_against_oracle(host(buf).astype(np.float64), rhs_np, c0, c1)


FRESH = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, {root!r})
from oracle import admm
from paper_2301_00406_gb300 import nlos
import ctypes
lib = nlos.load()
n, nt, c0, c1 = 64, 256, 2.5, 7.0
rhs_np = np.random.default_rng(3).standard_normal((n, n, nt))
s = torch.cuda.Stream()                       # created non-blocking by torch
with torch.cuda.stream(s):
    rhs = torch.tensor(rhs_np, dtype=torch.float32, device="cuda")
    x = torch.empty_like(rhs)
    st = lib.nlos_solve_static(n, n, nt, ctypes.c_void_p(rhs.data_ptr()), ctypes.c_void_p(x.data_ptr()), c0, c1,
                               ctypes.c_void_p(s.cuda_stream))
s.synchronize()
assert st == 0, nlos.last_error()
want = admm.fft_solve(rhs_np, c0, c1)
err = np.linalg.norm(x.cpu().numpy() - want) / np.linalg.norm(want)
print("fresh-process first call on a side stream: rel L2", err)
assert err < 1e-5
"""


def test_solve_static_first_call_in_fresh_process_on_side_stream():
    r = subprocess.run([sys.executable, "-c", FRESH.format(root=ROOT)], capture_output=True, text=True, timeout=300)
    print(r.stdout, r.stderr[-2000:])
    assert r.returncode == 0


def test_solve_static_rejects_grids_beyond_its_scratch():
    import torch
    from paper_2301_00406_gb300 import nlos
    lib = nlos.load()
    buf = torch.zeros(8, device="cuda")
    for n, nt in [(128, 64), (64, 1024), (48, 64), (32, 8)]:
        assert _static_solve(lib, n, nt, buf, buf, 1.0, 1.0) == -1
    assert "static" in nlos.last_error() or "powers of two" in nlos.last_error()
