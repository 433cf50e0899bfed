"""Host logic of bench.py without a GPU: the multi-rank timing aggregation on
two gloo ranks (the path torchrun takes for --gpus N, replicas only), the
reference arm's JSON line, and the roofline traffic bookkeeping."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    dist = bench.dist_init(world, use_cuda=False)
    bench.barrier(dist)
    t_max = bench.max_over_ranks(dist, 1.0 + rank)  # rank 1 is the slowest
    total = bench.sum_over_ranks(dist, 3.0)         # 3 trajectories per rank
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as fh:
        json.dump({"t_max": t_max, "total": total, "value": total / t_max}, fh)
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo(tmp_path):
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(2)]
    for r in res:
        assert r["t_max"] == 2.0 and r["total"] == 6.0 and r["value"] == 3.0


def test_single_rank_needs_no_process_group():
    assert bench.dist_init(1, use_cuda=False) is None
    assert bench.max_over_ranks(None, 4.5) == 4.5
    assert bench.sum_over_ranks(None, 2.0) == 2.0


def test_reference_arm_prints_one_json_line():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "trajectories/s" and d["higher_is_better"] is True
    cb = d["cpu_baseline"]
    assert d["value"] > 0 and cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert cb["single_thread"]["cores"] == 1 and cb["single_thread"]["value"] > 0
    assert cb["host"]["nproc"] == os.cpu_count() and cb["host"]["model"]
    assert d["arithmetic"]["forces"] == "f64 arithmetic" and d["arithmetic"]["solver"] == "fp64 CG"
    assert d["arithmetic"]["initial_guess"] == "zero"
    # the workload block is the one the GPU arm prints with the default arguments
    assert d["config"] == bench.config_block(bench.parse_args([]))
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["config"]["workload"] == "nf2_wilson_hmc_32x32x32x64"


def test_reference_arm_other_ranks_do_nothing():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_derived_trajectory_counts_every_part():
    sample = {"parts_s": {"cg_iteration": 1.0, "gauge_force": 10.0, "fermion_force": 100.0, "link_update": 1000.0},
              "scale": 2.0}
    # 16 Omelyan steps: 33 force evaluations, 32 link updates
    assert bench.derived_traj_s(sample, 7) == 2.0 * (7 + 33 * 110.0 + 32 * 1000.0)


def test_stored_traffic_is_dropped_when_the_kernel_changed(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic_dslash_f16n_32x32x32x64.txt").write_text(
        "# test\nkernel_source_sha=0000\ndram_bytes_per_launch=123\n")
    monkeypatch.setattr(bench, "HERE", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0000")
    assert bench.stored_traffic("dslash_f16n") == 123.0
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "ffff")
    assert bench.stored_traffic("dslash_f16n") is None
