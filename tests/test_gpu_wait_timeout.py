"""Failure detection without a GPU fault: a bounded mbarrier wait that nothing
completes gives up after its limit, the kernel reports NLOS_ERR_TIMEOUT
through device memory and returns, and the context stays usable (an
operator application afterwards still matches the FP64 oracle)."""

import time

import numpy as np
import pytest

from oracle import lct
from tests.gpu_util import dev, host, rel_l2

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_context_survives():
    import torch
    from paper_2301_00406_gb300 import nlos
    nlos.load()
    status = torch.full((1,), 12345, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nlos.selftest_wait_timeout(200, status)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    assert int(status.item()) == -6          # NLOS_ERR_TIMEOUT
    assert 0.19 < dt < 3.0, dt               # gave up after about its 200 ms limit

    # the context is intact: an operator application afterwards still matches the oracle
    n, nt, bw = 16, 128, 64e-12
    g = lct.Geometry(n, n, nt, bw)
    u = np.random.default_rng(5).random((n, n, nt))
    plan = nlos.Plan(n, n, nt, bw)
    got = host(nlos.forward_t(plan, dev(u), apply_mask=False))
    plan.close()
    assert rel_l2(got, lct.Operator(g).forward(u)) < 1e-5


def test_selftest_rejects_bad_arguments():
    import torch
    from paper_2301_00406_gb300 import nlos
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    for ms in (0, 5001):
        with pytest.raises(nlos.NlosError):
            nlos.selftest_wait_timeout(ms, status)
