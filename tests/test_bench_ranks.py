"""The benchmark's multi-process logic on CPU ranks (gloo, world size 2): the replicas'
step times reduce with a maximum and their particle counts with a sum, the reference arm
runs on rank 0 only, and the rank environment is read the way torchrun sets it."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      LOCAL_RANK=str(rank), WORLD_SIZE=str(world))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, lr, w = bench.dist_env()
        step_ms = 10.0 + 2.5 * rank   # rank 1 is the slow one
        parts = 3_000_000_000 + rank  # beyond 2^31: the sum must stay exact
        t, p = bench.reduce_ranks(torch, tdist, step_ms, parts, device="cpu")
        q.put((r, lr, w, t, p))
    finally:
        tdist.destroy_process_group()


def test_replica_reduction_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[:3] for o in out] == [(0, 0, 2), (1, 1, 2)]
    for o in out:
        assert o[3] == 12.5                       # max over ranks
        assert o[4] == 2 * 3_000_000_000 + 1       # sum over ranks, exact


def test_single_process_needs_no_collective():
    assert bench.reduce_ranks(torch, None, 7.0, 42) == (7.0, 42)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:  # never read on a non-zero rank
        pass

    assert bench.run_reference(Args(), {}) is None
    assert capsys.readouterr().out == ""


def test_ensemble_cpu_baseline_uses_every_thread():
    """The scan's oracle baseline steps one member per host thread concurrently and reports
    the aggregate rate with the thread count."""
    import bench

    r = bench.ensemble_cpu_baseline(4, budget_s=0.5)
    assert r["kind"] == "oracle" and r["unit"] == "particle-steps/s"
    assert 1 <= r["cores"] <= 4 and r["value"] > 0


def test_clock_samples_that_reject_a_timed_region():
    """A hardware or thermal slowdown, or an SM clock well below its maximum with no reason
    given (a leftover lock), rejects the timed region (bench.py measures it once more); a
    power cap is kept."""
    import bench

    ok = {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": []}
    assert not bench.clocks_rejected(ok)
    assert not bench.clocks_rejected(dict(ok, sm_mhz=1900.0, reasons=["sw_power_cap"]))
    assert bench.clocks_rejected(dict(ok, sm_mhz=1500.0))
    for r in ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"):
        assert bench.clocks_rejected(dict(ok, reasons=[r]))
    assert not bench.clocks_rejected({"sm_mhz": None, "sm_max_mhz": None,
                                      "reasons": ["nvidia-smi unavailable"]})
