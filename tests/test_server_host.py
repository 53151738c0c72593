"""Host-side failure handling of the serving runtime, without a GPU: invalid
arguments are refused at submit, and a job whose device set-up fails (here:
no CUDA device in this process) ends with an error status instead of
hanging; shutdown with a bounded wait returns."""

import numpy as np
import pytest


@pytest.fixture(scope="module")
def nlos():
    from paper_2301_00406_gb300 import build, nlos as mod
    build.build_library()
    mod.load()
    return mod


def test_server_rejects_bad_arguments(nlos):
    with pytest.raises(nlos.NlosError):
        nlos.Server(hbm_budget_bytes=0, max_slots=1)
    with pytest.raises(nlos.NlosError):
        nlos.Server(hbm_budget_bytes=1 << 30, max_slots=0)
    srv = nlos.Server(hbm_budget_bytes=1 << 30, max_slots=1)
    p = nlos.params_default(1)
    tau0 = np.zeros((12, 12, 64), np.float32)
    out = np.zeros_like(tau0)
    with pytest.raises(nlos.NlosError):
        srv.submit(12, 12, 64, 16e-12, p, tau0, out)      # nx not a power of two
    srv.close(timeout_s=5.0)


def test_failed_device_setup_is_reported(nlos):
    import torch
    if torch.cuda.is_available():
        pytest.skip("exercises the no-device failure path")
    srv = nlos.Server(hbm_budget_bytes=1 << 30, max_slots=1)
    p = nlos.params_default(1)
    p.iters = 2
    tau0 = np.zeros((8, 8, 16), np.float32)
    out = np.zeros_like(tau0)
    jid = srv.submit(8, 8, 16, 16e-12, p, tau0, out)
    with pytest.raises(nlos.NlosError) as e:
        srv.wait(jid, timeout_s=30.0)
    assert e.value.status in (-2, -3)
    assert srv.info()["failed"] == 1
    srv.close(timeout_s=5.0)
