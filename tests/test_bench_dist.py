"""The bench's host logic on CPU: the multi-rank path (two gloo ranks, as
replicas, each time their own work; the job's time is the slowest rank's and
its throughput is the units of all ranks over that time) and the read-back of
the plan tuner's choices for the bench line."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    r, w, _ = bench.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        t_max = bench.max_over_ranks(times[r], w, "cpu")
        out.put((r, t_max, bench.job_rate(50, w, t_max)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_report_slowest_time_and_total_units():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [40.0, 55.0]           # ms per rank
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for r, t_max, rate in got:
        assert t_max == 55.0
        assert rate == pytest.approx(2 * 50 / 0.055)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.job_rate(50, 1, 100.0) == pytest.approx(500.0)


def test_tuning_choices_read_back_for_the_geometry(tmp_path, monkeypatch):
    """The bench line's record of the plan tuner: the entries of this nt, the
    lateral solve's kernel of this plane size, nothing from other sizes."""
    import bench
    path = tmp_path / "tune"
    path.write_text("nlos-gb300 t-pass tuning v1\nsome GPU | 152 SMs | build\n"
                    "0 512 16384 8\n3 512 1024 260\n9 512 128 2\n9 512 64 1\n9 256 32 1\n4 256 1024 16\n")
    monkeypatch.setenv("NLOS_TUNE_CACHE", str(path))
    got = bench.tuning_choices(512, 128)
    assert got["lateral_solve"] == "half-warp transforms"
    assert got["tpass"] == [{"kind": "tfwd_rz", "columns": 16384, "cols_per_cta": 8, "batched_halves": False},
                            {"kind": "tinv_fit", "columns": 1024, "cols_per_cta": 4, "batched_halves": True}]
    assert [e["columns"] for e in bench.tuning_choices(512, 128, (16384,))["tpass"]] == [16384]
    assert bench.tuning_choices(256, 32)["lateral_solve"] == "shared-memory passes"
    monkeypatch.setenv("NLOS_TUNE_CACHE", "off")
    assert bench.tuning_choices(512, 128) is None
