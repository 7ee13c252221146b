"""Host-side logic of bench.py (no GPU): the reference arm's JSON line and rank
handling, and the multi-rank timing reduction over world_size-2 gloo ranks."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

SMALL = ["--impl", "reference", "--m", "512", "--n", "256", "--r1", "64", "--k", "16",
         "--cpu-rows", "64", "--steps", "1", "--warmup", "0"]


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + SMALL, env=env,
                          capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _run({"RANK": "0"})
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["unit"] == "ms" and d["higher_is_better"] is False and d["value"] > 0
    cb = d["cpu_baseline"]
    # two row samples, their difference extrapolated linearly in m
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and "64 and 128 of 512 rows" in cb["sample"]
    assert cb["value"] == d["value"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["h2d_bytes_per_step"] == 0
    assert e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_without_work():
    r = _run({"RANK": "1"})
    assert r.returncode == 0 and r.stdout.strip() == ""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank            # rank 1 is the slower one
        total = bench.max_over_ranks(ms, dist, "cpu")
        out[rank] = (total, bench.per_approximation_ms(total, 4, world))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    # both ranks see the slowest rank's time; 2 ranks x 4 steps share it
    assert res[0] == res[1] == (15.0, 15.0 / 8)


def test_protocol_summary_curves_and_time_to_target():
    recs = []
    for t in range(3):
        for q, (ms, err) in enumerate([(2.0, 0.5), (3.0, 0.08), (4.0, 0.05)]):
            recs.append({"method": "sketched", "l": 800, "q": q, "ms": ms + 0.1 * t, "err": err})
        for q, (ms, err) in enumerate([(2.5, 0.4), (3.5, 0.09)]):
            recs.append({"method": "sketched", "l": 1600, "q": q, "ms": ms, "err": err})
        for q, (ms, err) in enumerate([(5.0, 0.9), (9.0, 0.3)]):
            recs.append({"method": "classical", "l": 15000, "q": q, "ms": ms, "err": err})
    curves, best = bench.protocol_summary(recs, 0.1)
    assert [p[0] for p in curves["sketched:800"]] == [0, 1, 2]
    q1 = curves["sketched:800"][1]
    assert q1[1] == pytest.approx(3.1) and q1[2] == pytest.approx(0.08) and q1[3] == 3
    # the fastest iterate under the target, over every sketch size
    assert best["sketched"] == {"ms": pytest.approx(3.1), "err": pytest.approx(0.08), "l": 800, "q": 1}
    assert best["classical"] is None           # never reaches 0.1 within its iterates


def test_cpu_fit_extrapolates_only_the_row_linear_part(monkeypatch):
    # a fake oracle whose time is 100 ms of fixed work plus 2 ms per row: the fit
    # must return 100 + 2 m at any m, not the sample's time scaled by m / rows
    import argparse
    import numpy as np
    monkeypatch.setattr(bench, "cpu_oracle_ms", lambda A, a: 100.0 + 2.0 * A.shape[0])
    a = argparse.Namespace(m=65536)
    est, t1, t2, rows = bench.cpu_oracle_fit(np.zeros((4096, 8)), a)
    assert rows == 2048 and t1 == 100.0 + 2.0 * 2048 and t2 == 100.0 + 2.0 * 4096
    assert abs(est - (100.0 + 2.0 * 65536)) < 1e-9
