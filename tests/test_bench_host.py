"""Host-side logic of bench.py that needs no GPU: the oracle timing samples
and the reference arm's JSON line."""
import json
import os
import subprocess
import time
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_sample_shape_shrinks_only_for_large_workloads():
    assert bench._oracle_sample_shape(bench.WORKLOADS["ising-L32-h16-m4"], 12.0) == (16, 4)
    assert bench._oracle_sample_shape(bench.WORKLOADS["ising-L8-h4-m2"], 12.0) == (4, 2)
    assert bench._oracle_sample_shape(bench.WORKLOADS["ising-L128-h128-m32"], 12.0) == (2, 1)


def test_oracle_sample_stops_at_convergence():
    """Ising 8 x 8, 4 windows x 2 walkers, seed 0 converges after 63000 sweeps
    (the oracle's own run): a sample with no time limit runs exactly those
    630 blocks and counts at most every walker's attempts in each."""
    wl = bench.WORKLOADS["ising-L8-h4-m2"]
    att, el, blocks = bench._oracle_blocks(wl, 4, 2, 0, 1e9)
    assert blocks == 630
    assert 0 < att <= blocks * bench.SPE * 64 * 8
    assert att < blocks * bench.SPE * 64 * 8     # windows that finish early stop counting


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3", "--workload", "ising-L8-h4-m2"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "attempts/s" and line["value"] > 0
    assert line["cpu_baseline"]["cores"] == bench.host_cores() and line["cpu_baseline"]["kind"] == "oracle"
    assert line["cpu_baseline"]["value"] == line["value"] == line["e2e"]["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_latency_bound_is_read_from_the_committed_summary():
    assert 50.0 < bench.isolated_step_cycles() < 1000.0


def test_rates_microbenchmark_builds():
    import shutil

    import pytest

    if not (shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc")):
        pytest.skip("no CUDA toolkit")
    import ubench

    assert os.path.exists(ubench.build())


def test_all_cores_timing_fails_loudly_when_one_solve_fails(monkeypatch):
    """One failing oracle solve must end the all-cores sample with an error,
    not leave the others waiting at the start barrier."""
    import pytest

    real = bench._oracle_blocks

    def flaky(wl, h, m, seed, seconds, barrier=None):
        if seed == 1:
            raise ValueError("planted failure")
        return real(wl, h, m, seed, seconds, barrier)

    monkeypatch.setattr(bench, "_oracle_blocks", flaky)
    monkeypatch.setattr(bench, "host_cores", lambda: 3)
    with pytest.raises(RuntimeError, match="planted failure"):
        bench.oracle_rate_all_cores(bench.WORKLOADS["ising-L8-h4-m2"], 0, 0.5)


def test_fifo_latencies_follow_the_queue_by_hand():
    """One server, first come first served: arrivals 0, 1, 5 with services 3, 1, 2
    finish at 3, 4, 7, so the latencies are 3, 3, 2."""
    assert bench._fifo_latencies([0.0, 1.0, 5.0], [3.0, 1.0, 2.0]) == [3.0, 3.0, 2.0]
    assert bench._fifo_latencies([], []) == []


def test_served_stream_mix():
    """The served stream: one third of each model, each model's own sizes,
    q = 10 for Potts, request seed = index."""
    reqs = bench.served_requests(3000, 0)
    sizes = {m: set(s) for m, s, _ in bench.SERVED_MIX}
    counts = {m: 0 for m in sizes}
    for i, r in enumerate(reqs):
        assert r["seed"] == i and r["L"] in sizes[r["model"]]
        assert r["q"] == (10 if r["model"] == "potts" else 2)
        counts[r["model"]] += 1
    assert all(abs(c / 3000 - 1 / 3) < 0.04 for c in counts.values())
    assert bench.served_requests(50, 7) == bench.served_requests(50, 7)


def test_profile_traffic_only_for_the_profiled_source(tmp_path, monkeypatch):
    """roofline.traffic comes from the committed ncu summary only while its
    kernel_source_hash equals the hash of the current sweep sources, and only for
    the profiled workload and sweep form; else it is null."""
    f = tmp_path / "summary.txt"
    f.write_text("kernel_source_hash = %s\ndram_bytes_per_launch = 1234\n" % bench.kernel_source_hash())
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", str(f))
    assert bench.traffic_from_profile(bench.DEFAULT_WORKLOAD, 2) == 1234.0
    assert bench.traffic_from_profile(bench.DEFAULT_WORKLOAD, 0) is None
    assert bench.traffic_from_profile("ising-L128-h128-m32", 2) is None
    f.write_text("kernel_source_hash = 0000000000000000\ndram_bytes_per_launch = 1234\n")
    assert bench.traffic_from_profile(bench.DEFAULT_WORKLOAD, 2) is None


def test_plain_stream_threads_follow_arrivals_and_the_concurrency_limit(monkeypatch):
    """The measured plain arm of the served-stream benchmark: each request
    starts at its arrival on its own thread, at most `concurrency` at once;
    latency = end - arrival.  With one at a time it is the FIFO queue."""
    import bench

    def fake(rewl, r, stop=None):
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < r["dur"]:
            if stop is not None and stop.is_set():
                return (None, 5)
            time.sleep(0.005)
        return (r["seed"], 10)

    monkeypatch.setattr(bench, "_plain_request", fake)
    reqs = [dict(seed=k, dur=d) for k, d in enumerate([0.30, 0.10, 0.20])]
    arrivals = [0.0, 0.05, 0.50]
    lat, res, wall = bench.run_plain_stream(None, reqs, arrivals, 1)
    want = bench._fifo_latencies(arrivals, [0.30, 0.10, 0.20])
    assert all(abs(a - b) < 0.05 for a, b in zip(lat, want)), (lat, want)
    assert [r[0] for r in res] == [0, 1, 2]
    lat2, _, _ = bench.run_plain_stream(None, reqs, arrivals, 3)   # no queueing: latency = own duration
    assert all(abs(a - d) < 0.05 for a, d in zip(lat2, [0.30, 0.10, 0.20])), lat2
    s = bench._summary(lat2 + [None], list(res) + [(None, 0)], 1.0)
    assert s["completed"] == 3 and s["unfinished"] == 1 and s["attempts_per_s"] == 30.0
    # stopped after 0.35 s: the 0.3 s request finishes, the one queued behind it (one at a time,
    # running from 0.3 s) is abandoned, the one arriving at 0.5 s never starts
    lat3, res3, wall3 = bench.run_plain_stream(None, reqs, arrivals, 1, stop_after=0.35)
    assert lat3[0] is not None and lat3[1] is None and lat3[2] is None
    assert res3[1] == (None, 5) and res3[2] == (None, 0) and abs(wall3 - 0.35) < 0.05
