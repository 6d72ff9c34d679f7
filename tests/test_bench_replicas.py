"""bench.py's host logic on CPU.  With N > 1 ranks (replicas: one
independent chain per rank, no data-path collective), on two gloo ranks: the
timing taken is the slowest rank's, the rate counts every rank's
trajectories, the chains are seeded apart, and the reference arm runs on
rank 0 only.  On one rank: the reference arm's JSON line (the oracle on the
host cores) and the refusal of fewer than three warm-up steps."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, os.environ["BENCH_ROOT"])
import torch.distributed as dist
dist.init_process_group("gloo", init_method="env://")
import bench
rank, world = dist.get_rank(), dist.get_world_size()
ms = 100.0 + 50.0 * rank                    # this rank's timed region
slowest = bench.max_over_ranks(ms, world, "cpu")
print(json.dumps({"rank": rank, "slowest_ms": slowest, "rate": bench.job_rate(world, 4, slowest / 1e3),
                  "seed": bench.replica_seed(0x5A0002, rank)}))
dist.barrier()
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, world, port):
    env = dict(os.environ)
    env.update({"RANK": str(rank), "LOCAL_RANK": str(rank), "WORLD_SIZE": str(world), "MASTER_ADDR": "127.0.0.1",
                "MASTER_PORT": str(port), "BENCH_ROOT": ROOT})
    return env


def test_two_gloo_ranks_take_the_slowest_rank_and_count_every_rank():
    port = _free_port()
    procs = [subprocess.Popen([sys.executable, "-c", RANK_SCRIPT], env=_env(r, 2, port), stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for r in range(2)]
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=300)
        assert p.returncode == 0, err[-2000:]
        outs.append(json.loads(out.strip().splitlines()[-1]))
    outs.sort(key=lambda o: o["rank"])
    assert all(o["slowest_ms"] == 150.0 for o in outs)
    assert all(abs(o["rate"] - 2 * 4 / 0.150 * 3600.0) < 1e-9 for o in outs)
    assert outs[0]["seed"] != outs[1]["seed"]


def test_reference_arm_prints_on_rank_zero_only():
    """Under torchrun every rank but 0 exits 0 without work or output."""
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3"], env=_env(1, 2, _free_port()), capture_output=True,
                       text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""


def test_reference_arm_prints_the_contract_line():
    """bench.py --impl reference on one rank: one JSON line with the metric,
    a positive rate from the oracle on the host cores, its cpu_baseline
    record, an e2e record without copies, and the GPU arm's workload."""
    env = dict(os.environ)
    for k in ("RANK", "LOCAL_RANK", "WORLD_SIZE"):
        env.pop(k, None)
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == "trajectories/hour"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 3
    assert d["config"] == bench.workload_config(1)
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "trajectories/hour", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_fewer_than_three_warmup_steps_are_refused():
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--warmup", "2"],
                       capture_output=True, text=True, timeout=300)
    assert p.returncode == 2 and "--warmup" in p.stderr


def test_clock_summary_keeps_the_timed_window():
    """Samples taken before the timed region (the sampler's start-up) are left
    out when the window holds any; throttle reasons are those seen inside."""
    import bench
    c = bench.ClockSampler(0)
    c.lines = [(0.5, "900, 2070, 0x0, Not Active, Not Active, Not Active, Not Active"),
               (1.0, "2070, 2070, 0x0, Not Active, Not Active, Not Active, Active"),
               (2.0, "2070, 2070, 0x0, Not Active, Not Active, Not Active, Not Active")]
    c.window = (0.9, 2.5)
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["samples"] == 2 and s["reasons"] == ["sw_power_cap"]
    c.window = (5.0, 6.0)        # no sample inside: all of them
    assert c.summary()["samples"] == 3
