"""The multi-rank path of bench.py on CPU (gloo, world size 2): replicas are
timed per rank and the whole-job rate divides every rank's iterations by the
slowest rank's time (no collective on the data path)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp        # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, local_ms, q):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        q.put((rank, bench.whole_job_rate(local_ms[rank], 7200, world, dist, "cpu")))
    finally:
        dist.destroy_process_group()


def test_whole_job_rate_takes_the_slowest_rank():
    world, port = 2, _free_port()
    local_ms = [100.0, 150.0]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, local_ms, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        ms_max, value = res[r]
        assert ms_max == 150.0
        assert value == pytest.approx(2 * 7200 / 0.150)


def test_whole_job_rate_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.whole_job_rate(200.0, 7200, 1)
    assert ms == 200.0 and value == pytest.approx(36000.0)


def test_roofline_entry_arithmetic():
    # achieved = algorithmic bytes per launch / launch time; frac against the
    # peak; traffic only where a capture of the same kernel and tile exists
    sys.path.insert(0, ROOT)
    import bench
    algo = bench.stage_bytes(3, 1024, 50_000, 200, 90_000, 27_000, 128)
    assert algo["scan_phase3"] == 3 * (10 * 1024 * 1024 + 12 * 128 * 1024)
    assert algo["gather_move"] == 3 * 48 * 50_000
    batches = {"chain3": dict(algo=algo, stages={"scan_phase3": 0.02, "scan_phase1": 0.01},
                              tile=dict(band_rows=8, cols_per_thread=0, threads=256), per_step=1200)}
    pk = {"hbm_gbs": 6788.3}
    r = bench.roofline(batches, "chain3", "scan_phase3", pk)
    assert r["achieved"] == pytest.approx(algo["scan_phase3"] / 0.02e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    # scan phase 3 of this tile changed after its capture (label copies issued
    # before the launch wait): no traffic until it is captured again
    assert r["traffic"] is None
    assert bench.roofline(batches, "chain3", "scan_phase1", pk)["traffic"] == \
        bench.TRAFFIC[("chain3", "scan_phase1", 8, 0, 256)]
    # no capture of this tile: no traffic
    batches["chain3"]["tile"] = dict(band_rows=16, cols_per_thread=0, threads=256)
    assert bench.roofline(batches, "chain3", "scan_phase1", pk)["traffic"] is None
