"""The multi-rank (N > 1) path of bench.py on CPU: world_size-2 gloo process group,
barrier + max over ranks, whole-job value = all ranks' solves / slowest rank's time,
and the reference arm printing only on rank 0."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    per_rank_ms = [120.0, 250.0][rank]
    dist.barrier()
    m = bench.max_over_ranks(per_rank_ms)
    out.put((rank, m, bench.whole_job_rate(world, 10, m)))
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, rate in res:
        assert m == 250.0                      # the slowest rank decides
        assert abs(rate - 2 * 10 / 0.25) < 1e-9  # 2 replicas x 10 solves / 0.25 s


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.whole_job_rate(1, 4, 500.0) == 8.0


@pytest.mark.slow
def test_reference_arm_prints_on_rank_zero_only(tmp_path):
    # torchrun with 2 CPU ranks: only rank 0 prints the JSON line; rank 1 exits 0 without work
    env = dict(os.environ, PYTHONPATH=ROOT)
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=600, cwd=str(tmp_path))
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0


def test_reference_arm_json_line(monkeypatch, capsys):
    # the reference arm's JSON line (the oracle's own solver is replaced by a stand-in
    # that takes a known time per call, so only the plumbing and arithmetic run)
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    from oracle import iterations as oit
    calls = []

    def fake(p, lap, tol=0.0, max_it=0):
        calls.append(max_it)
        return None, max_it

    monkeypatch.setattr(oit, "fpsa_source_iteration", fake)
    for v in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(v, raising=False)
    args = argparse.Namespace(steps=2, warmup=3, gpus=1, laplacian="wfd", precision="mixed")
    bench.run_reference(args)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "solves/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["cpu_baseline"]["value"] == line["value"] == line["e2e"]["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["config"]["workload"].startswith("precision_srk_slab")
    assert line["config"] == bench.run_config(args, 1)  # the GPU arm's config object
    assert calls == [3, 5] * (args.warmup + args.steps)  # setup + 3 and 5 iterations per step
