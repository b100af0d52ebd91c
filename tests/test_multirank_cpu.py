"""The N > 1 path of the bench on the host: two gloo ranks (CPU, 127.0.0.1).

Each rank runs its own replica of the workload (the path shards into independent problems, so
there is no data-path collective); the only exchange is the step time, reduced to the slowest
rank's, and the whole-job rate counts every rank's units. The reference arm does its work on
rank 0 only; other ranks return without work.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, world)          # rank 1 is the slower one
        rate = bench.job_throughput(1000, world, ms)
        torch.distributed.barrier()
        out.put((rank, ms, rate))
    finally:
        torch.distributed.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_slowest_and_count_all_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]                       # max over ranks
    assert all(abs(r[2] - 2 * 1000 / 15e-3) < 1e-6 for r in res)     # world x units / slowest time


def test_single_rank_is_unchanged():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_throughput(100, 1, 2.0) == 100 / 2e-3


def test_reference_arm_other_ranks_do_no_work(capsys):
    import argparse
    import bench
    args = argparse.Namespace(config="stokes2d", pad=1, steps=1, warmup=0, gpus=2)
    assert bench.run_reference(args, rank=1, world=2) is None
    assert capsys.readouterr().out == ""


def test_reference_arm_prints_one_contract_line(capsys, monkeypatch):
    """Rank 0 of the reference arm times the oracle on the host and prints one JSON line with
    the bench contract's keys (the oracle's sample shortened here to keep the test quick)."""
    import argparse
    import json
    import bench
    full = bench.cpu_oracle_sample
    monkeypatch.setattr(bench, "cpu_oracle_sample",
                        lambda cfg, pts, seconds, seed=1: full(cfg, pts, 0.01, seed))
    args = argparse.Namespace(config="stokes2d", pad=1, steps=2, warmup=1, gpus=1)
    bench.run_reference(args, rank=0, world=1)
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1
    assert d["value"] > 0 and d["unit"] == "points/s" and d["higher_is_better"] is True
    assert d["config"]["workload"].startswith("stokes2d")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "points/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_cpu_oracle_pool_matches_one_process():
    """The bench's all-core CPU baseline (spawned processes, each rebuilding the sea from its seed)
    returns exactly the single-process oracle's values at the sampled points."""
    import numpy as np
    import bench
    from oracle import modal
    from wavegen import configs
    cfg = configs.jonswap3d(mesh_dims=(4, 8, 4))
    pts = configs.mesh_points(cfg["mesh"])[:200]
    rate, n, vals, idx, cores = bench.cpu_oracle_pool("jonswap3d", len(cfg["z_levels"]),
                                                      cfg["t_query"], pts, 0.3, 2)
    assert cores == 2 and n == len(idx) >= 2 and rate > 0
    ref = modal.fields_at_points(modal.propagate(cfg["sea"], cfg["t_query"]), pts[idx].astype(np.float64))
    for k in ("eta", "u", "v", "w", "p"):
        np.testing.assert_allclose(vals[k], ref[k], rtol=1e-12, atol=1e-12)
