"""Host-side helpers of bench.py on CPU: the traffic figures read from profiles/ (keyed by the
kernel sources' hash, so a changed kernel reads as unmeasured), the CPU model string, the
single-thread oracle timing in a child process, and the reference arm's JSON line (the
oracle timed on a small sample with the same workload label and core as the GPU arm)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_kernel_source_tag_tracks_the_sources():
    t1 = bench.kernel_source_tag("pass_tc3.cu", "tc_common.cuh")
    t2 = bench.kernel_source_tag("pass_tc3.cu", "tc_common.cuh")
    t3 = bench.kernel_source_tag("pass_tc.cu", "tc_common.cuh")
    assert t1 == t2 and t1 != t3 and len(t1) == 10


def test_traffic_lines_of_the_profiles_parse():
    """Every `traffic_bytes_per_launch` line of the committed ncu summaries names a kernel,
    dtype, size and source hash and gives a positive byte count that the bench can read
    back; an unknown hash reads as unmeasured."""
    import re
    d = os.path.join(ROOT, "profiles")
    keys = []
    for nm in sorted(os.listdir(d)):
        with open(os.path.join(d, nm)) as f:
            for line in f:
                mt = re.match(r"\s*traffic_bytes_per_launch\s+(\S+)\s+(\S+)", line)
                if mt:
                    pat = r"[a-z0-9_]+/[a-z0-9]+/[0-9a-z]+(/l[0-9]+)?/src-[0-9a-f]{10}"
                    assert re.fullmatch(pat, mt.group(1)), mt.group(1)
                    assert float(mt.group(2)) > 0
                    keys.append(mt.group(1))
    assert keys
    for k in keys:
        assert bench.traffic_from_profiles(k) > 0
    assert bench.traffic_from_profiles("pass_tc3_kernel/f32/20000x20000/l120/src-0000000000") is None


def test_cpu_model_is_a_string():
    s = bench.cpu_model()
    assert isinstance(s, str) and s


def test_single_thread_oracle_timing_runs_in_a_child():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((300, 200))
    phi = rng.standard_normal((200, 20))
    t = bench.oracle_single_thread_time(A, phi, {"dtype": "f32", "k": 10, "l": 20, "q": 1}, "sketch")
    assert t is not None and 0.0 < t < 60.0


def test_reference_arm_line():
    """`--impl reference` prints one JSON line: the oracle's rate on the default workload with
    the GPU arm's workload label and core, a cpu_baseline describing the run and an e2e with no
    host copies."""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--m", "1200", "--n", "1000"],
                         capture_output=True, text=True, timeout=600, check=True).stdout
    line = [x for x in out.splitlines() if x.startswith("{")][-1]
    d = json.loads(line)
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "solves/s"
    assert d["config"]["core"] == "sketch" and "sketch core" in d["config"]["workload"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["cpu_model"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
