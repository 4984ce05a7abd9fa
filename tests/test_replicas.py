"""bench.py's multi-process path on CPU: two gloo ranks (replicas), the
max-over-ranks job time and the whole-job aggregate."""
import json
import os
import socket

import pytest
import torch.multiprocessing as mp

from tests import _replica_worker


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_replicas(tmp_path):
    world = 2
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_replica_worker.run, args=(r, world, port, str(tmp_path))) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
    for p in procs:
        if p.is_alive():
            p.kill()
            pytest.fail("a replica did not finish")
        assert p.exitcode == 0
    res = [json.load(open(os.path.join(tmp_path, f"rank{r}.json"))) for r in range(world)]
    for r, d in enumerate(res):
        assert d["rank"] == r and d["world"] == world and d["local"] == r and d["backend"] == "gloo"
        assert d["ms"] == 15.0                      # the slowest rank (10 + 5 * 1 ms)
        assert abs(d["value"] - 2 * 2.0e12 / 15e-3 / 1e12) < 1e-9


def test_single_process_defaults(monkeypatch):
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_init() == (0, 1, 0)
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert abs(bench.job_tflops(1.0e12, 10.0, 1) - 100.0) < 1e-12
