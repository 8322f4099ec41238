"""Host-side logic of bench.py that needs no GPU: the reference arm (the
oracle timed on the host cores) and its launch contract, the max-over-ranks
reduction of replica timings over a two-rank gloo group, the predicate that
says when the Gram is grouped by the leading index, and the x2 ladder of
sample counts for the 1.01x loss target (its stopping rule, and the oracle's
ladder on the small workload)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import synth  # noqa: E402

SMALL = "dense3_64_r4_f64"


def _run(args, env_extra=None, timeout=300):
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT"):
        env.pop(k, None)
    env.update(env_extra or {})
    return subprocess.run([sys.executable] + args, cwd=ROOT, env=env, capture_output=True,
                          text=True, timeout=timeout)


def _json_lines(out):
    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_reference_arm_line():
    r = _run(["bench.py", "--impl", "reference", "--workload", SMALL, "--steps", "2",
              "--warmup", "1"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    ln = lines[0]
    assert ln["impl"] == "reference"
    assert ln["metric"] == bench.METRIC and ln["unit"] == "ms"
    assert ln["higher_is_better"] is False
    assert ln["steps"] == 2 and ln["warmup"] == 1 and ln["n_gpus"] == 1
    assert ln["value"] > 0 and ln["ms_per_step"] == ln["value"]
    assert ln["config"]["workload"] == SMALL
    cb = ln["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == ln["value"] and cb["cores"] >= 1
    assert cb["sample"]
    e2e = ln["e2e"]
    assert e2e["value"] == ln["value"] and e2e["unit"] == "ms"
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert ln["oracle_exact"]["ms"] > 0 and ln["oracle_exact"]["sample"]
    # the line is timed at the sample count its own ladder finds for the 1.01x target
    lad = ln["m_ladder"]
    assert lad["rows"] and lad["rows"][0]["m"] == ln["config"]["m_workload"]
    assert ln["config"]["m"] == (lad["m_star"] or ln["config"]["m_workload"])
    if lad["m_star"]:
        assert lad["rows"][-1]["median_ratio"] <= bench.LADDER_TARGET


def test_oracle_exact_timing_skips_the_observed_entry_gram():
    w = synth.WORKLOADS["missing3_1024_r16_f32"]
    ms, sample = bench.oracle_exact_timing(w, {"keys": None}, None)
    assert ms is None and sample.startswith("not run")


def test_reference_arm_other_ranks_exit_without_work():
    r = _run(["bench.py", "--impl", "reference", "--workload", SMALL, "--steps", "1",
              "--warmup", "1", "--gpus", "2"], {"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert _json_lines(r.stdout) == []


def test_reference_arm_under_torchrun_two_ranks():
    port = _free_port()
    r = _run(["-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
              "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py",
              "--impl", "reference", "--workload", SMALL, "--gpus", "2", "--steps", "1",
              "--warmup", "1"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1                      # rank 0 alone prints
    assert lines[0]["n_gpus"] == 2 and lines[0]["impl"] == "reference"


def _max_worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r times [1 + r, 10 - r, 5]: the job's time is the slowest replica's
        got = bench.max_over_ranks([1.0 + rank, 10.0 - rank, 5.0], "cpu")
        q.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_two_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_max_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0] == res[1] == [2.0, 10.0, 5.0]


@pytest.mark.parametrize("name,expect", [
    ("dense3_64_r4_f64", False),        # d / R_1 = 16
    ("dense3_512_r8_f32", False),       # d / R_1 = 64
    ("dense4_128_r8_f32", True),        # d / R_1 = 512, I_1 = 128
    ("missing3_1024_r16_f32", True),    # d / R_1 = 256, I_1 = 1024, A^(1) 64 KB as FP32
])
def test_grouped_gram_predicate(name, expect):
    assert bench.grouped_gram(synth.WORKLOADS[name]) is expect


def test_grouped_gram_predicate_limits():
    class W:
        def __init__(self, dims, ranks):
            self.dims, self.ranks = dims, ranks
            self.d = 1
            for r in ranks:
                self.d *= r
    assert not bench.grouped_gram(W((40, 40), (16, 16)))            # order 2
    assert not bench.grouped_gram(W((40, 40, 40), (3, 16, 16)))     # R_1 not a power of two
    assert not bench.grouped_gram(W((40, 40, 40), (32, 8, 16)))     # R_1 > 16
    assert bench.grouped_gram(W((40, 40, 40), (4, 16, 8)))          # d / R_1 = 128
    assert not bench.grouped_gram(W((40, 40, 40), (4, 8, 8)))       # d / R_1 = 64
    # at most 8192 (segment, tile) partials: d / R_1 = 512 has 3 upper tiles
    assert bench.grouped_gram(W((2730, 40, 40), (8, 16, 32)))
    assert not bench.grouped_gram(W((2731, 40, 40), (8, 16, 32)))
    # A^(1) in FP32 within 200 KB of shared memory
    assert bench.grouped_gram(W((3200, 40, 40), (16, 16, 16)))
    assert not bench.grouped_gram(W((3201, 40, 40), (16, 16, 16)))


@pytest.mark.parametrize("name,m,expect", [
    ("dense3_512_r8_f32", 100000, True),            # d / R_1 = 64: the narrow grouped Gram
    ("dense3_512_r8_f32", 1000, False),             # fewer than 2 I_1 rows
    ("dense4_128_r8_f32", 800000, False),           # d / R_1 = 512: the wide grouped Gram
    ("dense3_64_r4_f64", 2000, True),               # d / R_1 = 16
])
def test_narrow_gram_predicate(name, m, expect):
    assert bench.narrow_gram(synth.WORKLOADS[name], m) is expect


def test_narrow_gram_predicate_limits():
    class W:
        def __init__(self, dims, ranks):
            self.dims, self.ranks = dims, ranks
            self.d = 1
            for r in ranks:
                self.d *= r
    assert not bench.narrow_gram(W((40, 40), (8, 8)), 10 ** 5)              # order 2
    assert not bench.narrow_gram(W((40, 40, 40), (3, 4, 4)), 10 ** 5)       # R_1 not a power of two
    assert not bench.narrow_gram(W((40, 40, 40), (1, 8, 8)), 10 ** 5)       # R_1 = 1
    assert bench.narrow_gram(W((40, 40, 40), (16, 8, 8)), 10 ** 5)          # d / R_1 = 64
    assert not bench.narrow_gram(W((40, 40, 40), (2, 8, 16)), 10 ** 5)      # d / R_1 = 128
    assert bench.narrow_gram(W((3072, 40, 40), (8, 8, 8)), 6144)             # m = 2 I_1
    assert not bench.narrow_gram(W((3072, 40, 40), (8, 8, 8)), 6143)
    assert not bench.narrow_gram(W((3073, 40, 40), (8, 8, 8)), 10 ** 6)     # A^(1) over 96 KB


def test_ladder_helper_doubles_m_until_the_median_meets_the_target():
    calls = []

    def ratio_of(m, s):
        calls.append((m, s))
        return 1.0 + 50.0 / m + 1e-4 * s          # median over s = 0..9: 1 + 50/m + 4.5e-4
    rows, m_star = bench._ladder(ratio_of, 1000)
    assert [r["m"] for r in rows] == [1000, 2000, 4000, 8000]
    assert m_star == 8000 and rows[-1]["median_ratio"] <= bench.LADDER_TARGET
    assert all(r["median_ratio"] > bench.LADDER_TARGET for r in rows[:-1])
    assert len(calls) == 4 * bench.LADDER_SEEDS
    rows, m_star = bench._ladder(lambda m, s: 1.5, 10)   # never met within the ladder
    assert m_star is None and len(rows) == bench.LADDER_STEPS + 1


def test_m_ladder_reference_small_workload():
    r = _run(["bench.py", "--impl", "reference", "--m-ladder", "--workload", SMALL])
    assert r.returncode == 0, r.stderr[-2000:]
    (ln,) = _json_lines(r.stdout)
    assert ln["mode"] == "m_ladder" and ln["impl"] == "reference" and ln["workload"] == SMALL
    ms = [row["m"] for row in ln["ladder"]]
    assert ms[0] == synth.WORKLOADS[SMALL].m and all(b == 2 * a for a, b in zip(ms, ms[1:]))
    assert ln["ladder"][-1]["median_ratio"] <= 1.01 and ln["m_star"] == ms[-1]
    assert all(row["median_ratio"] >= 1.0 for row in ln["ladder"])
