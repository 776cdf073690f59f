#!/usr/bin/env python3
"""Benchmark of the GB300 REWL library: spin-flip attempts per second of the
whole REWL pipeline (WL sweeps, exchange rounds, flatness checks and merges)
on the Ising 32 x 32 workload with 16 windows x 4 walkers, ln f -> 1e-8.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

One step = one flatness period of the solve: 1000 sweeps of every active
walker (10 blocks of 100 sweeps, each followed by an exchange round) and one
flatness check / merge.  Inputs are resident on the device when the timed
region starts; L2 is flushed (256 MiB written) between timed steps, outside
the per-step CUDA events.  Under torchrun every rank runs an independent
replica with its own seed (the method shards by independent solves; there is
no data-path collective), value = all attempts / max time over ranks.

Prints one JSON line (rank 0).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

def sites(wl):
    """Sites of a workload's lattice: L^2, or L^3 on the cube."""
    return wl["L"] ** 3 if wl["model"] == "ea3d" else wl["L"] ** 2


WORKLOADS = {
    "ising-L32-h16-m4": dict(model="ising", L=32, q=2, h=16, m=4, lnf_final=1e-8,
                             desc="2D Ising L=32 periodic J=1; 16 windows at 75% overlap x 4 walkers (64 walkers); "
                                  "flatness 0.8 checked every 1000 sweeps; ln f 1 -> 1e-8; swaps every 100 sweeps"),
    "ising-L8-h4-m2": dict(model="ising", L=8, q=2, h=4, m=2, lnf_final=1e-6,
                           desc="2D Ising L=8; 4 windows at 75% overlap x 2 walkers; ln f 1 -> 1e-6"),
    "potts-q10-L32-h32-m16": dict(model="potts", L=32, q=10, h=32, m=16, lnf_final=1e-8,
                                  desc="2D q=10 Potts L=32; 32 windows at 75% overlap x 16 walkers (512 walkers); "
                                       "ln f 1 -> 1e-8"),
    "ea3d-L12-h16-m4": dict(model="ea3d", L=12, q=2, h=16, m=4, lnf_final=1e-6,
                            desc="3D +-J spin glass 12x12x12 periodic, couplings +-1 at p=1/2 from the seed; "
                                 "16 windows at 75% overlap x 4 walkers; ln f 1 -> 1e-6"),
    "ising-L128-h128-m32": dict(model="ising", L=128, q=2, h=128, m=32, lnf_final=1e-6,
                                desc="2D Ising L=128; 128 windows at 75% overlap x 32 walkers (4096 walkers); "
                                     "ln f 1 -> 1e-6"),
}
DEFAULT_WORKLOAD = "ising-L32-h16-m4"
OVERLAP, FLATNESS, SPE, SPF = 0.75, 0.8, 100, 1000
METRIC = "spin-flip attempts/s (REWL: WL sweeps + exchange + flatness/merge)"
# Integer operations of one WL trial, counted as the hardware issues them
# (a 32x32->64 multiply and a three-input XOR are one instruction each):
# Philox4x32-10 10 x (2 wide multiplies + 2 XOR3) = 40 and its counter 2;
# site, row and column 3; ln u from two words (bits, convert, logf, scale,
# convert) 10; the neighbourhood (periodic indices 8, addresses 10, five
# loads, bit extraction 10, bond count 8) 41; energy change, bin and window
# test 3; shadow load and the fixed-point test 7; configuration, shadow and
# bin updates and counters 10.  About 116, within the 100-125 that an
# independent itemisation of a 2D Ising trial gives; 112 is used.
OPS_PER_ATTEMPT = 112
N_SM = 152
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "k_sweep_ising_L32_h16_m4.txt")


SWEEP_SOURCES = ("rewl_device.cuh", "rewl_kernels.cu", "rewl_layout.h")


def kernel_source_hash():
    """Hash of the sources the sweep kernel is compiled from."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1305_5615_gb300", "csrc")
    for f in SWEEP_SOURCES:
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


UBENCH_SUMMARY = os.path.join(ROOT, "profiles", "ubench_pipe_rates_and_wl_step_latency.txt")


def measured_int_rate():
    """The highest measured integer issue rate (lane-ops per clock per SM) of
    the microbenchmark's integer mixes -- the Philox round's 32x32->64
    multiply + XOR3, 32-bit multiply + XOR3 + add, add3 + XOR3 -- from the
    committed summary; None if absent.  Taking the fastest mix as the peak
    keeps the roofline fraction conservative."""
    if not os.path.exists(UBENCH_SUMMARY):
        return None
    rates = []
    for line in open(UBENCH_SUMMARY):
        if line.startswith("integer mix"):
            try:
                rates.append(float(line.split("lane-ops")[0].split()[-1]))
            except (IndexError, ValueError):
                pass
    return max(rates) if rates else None


def measured_philox_rate():
    """Measured Philox4x32-10 calls per clock per SM (microbenchmark summary)."""
    if not os.path.exists(UBENCH_SUMMARY):
        return None
    for line in open(UBENCH_SUMMARY):
        if line.startswith("Philox4x32-10"):
            try:
                return float(line.split("calls/clk/SM")[0].split()[-1])
            except (IndexError, ValueError):
                return None
    return None


def isolated_step_cycles():
    """Cycles per trial of the sequential WL step run on its own (the
    microbenchmark's dependency chain on the int64 shadow), from the committed
    summary; None if absent."""
    if not os.path.exists(UBENCH_SUMMARY):
        return None
    for line in open(UBENCH_SUMMARY):
        if line.startswith("int64 shadow, dependency chain only"):
            try:
                return float(line.split()[5])
            except (IndexError, ValueError):
                return None
    return None


def traffic_from_profile(workload, variant):
    """DRAM bytes per sweep launch from the committed ncu summary, if it was
    taken on the current kernel source, for this workload and sweep form
    (the ring form on the default workload); else None."""
    if workload != DEFAULT_WORKLOAD or variant != 2 or not os.path.exists(PROFILE_SUMMARY):
        return None
    kv = {}
    for line in open(PROFILE_SUMMARY):
        if "=" in line and not line.startswith("#"):
            k, v = line.split("=", 1)
            kv[k.strip()] = v.strip()
    if kv.get("kernel_source_hash") != kernel_source_hash():
        return None
    try:
        return float(kv["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p))
        except Exception:
            return {}
    return {}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for i, n in enumerate(names):
                    if r[5 + i].lower().startswith("active"):
                        reasons.add(n)
            except (IndexError, ValueError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def replica_seed(base, rank):
    """Seed of the replica on `rank`: independent solves, one per rank."""
    return base + rank


def aggregate_replicas(t_local, att_local, world, device="cuda"):
    """Whole-job throughput of independent replicas: attempts of all ranks /
    the longest rank's time (max-over-ranks timing)."""
    if world <= 1:
        return att_local / t_local, t_local, att_local
    import torch
    import torch.distributed as dist

    tt = torch.tensor([t_local], dtype=torch.float64, device=device)
    aa = torch.tensor([att_local], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    dist.all_reduce(aa, op=dist.ReduceOp.SUM)
    return float(aa.item()) / float(tt.item()), float(tt.item()), float(aa.item())


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


ORACLE_TRIALS_PER_S = 2.5e7   # rough single-core oracle speed, to size the sample


def _oracle_sample_shape(wl, seconds):
    """Windows and walkers of the oracle's timing sample: the workload itself,
    or the same lattice with 2 windows x 1 walker when one exchange block of
    the whole workload would take much longer than `seconds` (the oracle's
    cost per trial does not depend on the walker count)."""
    h, m = wl["h"], wl["m"]
    if h * m * SPE * sites(wl) / ORACLE_TRIALS_PER_S > 2 * seconds:
        h, m = 2, 1
    return h, m


def _oracle_blocks(wl, h, m, seed, seconds, barrier=None):
    """Creates one oracle solve (entry walk untimed), optionally waits at
    `barrier`, then runs whole exchange blocks for about `seconds`.
    Returns (attempts, seconds, blocks)."""
    from oracle import OracleREWL

    O = OracleREWL(wl["model"], wl["L"], h, OVERLAP, m, FLATNESS, wl["lnf_final"], seed, q=wl["q"],
                   sweeps_per_exchange=SPE, sweeps_per_flat_check=SPF)
    if barrier is not None:
        barrier.wait()
    t0 = time.perf_counter()
    blocks, att = 0, 0
    while True:
        active = m * sum(1 for d in O.windows()["done"] if not d)  # walkers of windows still running
        if active == 0:
            break
        O.run_blocks(1)
        blocks += 1
        att += active * SPE * O.N
        if time.perf_counter() - t0 >= seconds:
            break
    return att, time.perf_counter() - t0, blocks


def oracle_rate(wl, seed, seconds):
    """Single-threaded oracle attempts/s on the workload, for about `seconds`
    of CPU work (whole exchange blocks; entry walk excluded).  Returns (rate,
    blocks, seconds, walkers sampled)."""
    h, m = _oracle_sample_shape(wl, seconds)
    att, el, blocks = _oracle_blocks(wl, h, m, seed, seconds)
    return att / el, blocks, el, h * m


def host_cores():
    return os.cpu_count() or 1


def _run_threads(fn, n):
    th = [threading.Thread(target=fn, args=(k,)) for k in range(n)]
    for t in th:
        t.start()
    for t in th:
        t.join()


def oracle_rate_all_cores(wl, seed, seconds):
    """P = host_cores() independent oracle solves (seeds seed .. seed+P-1),
    one thread each, run at the same time: aggregate attempts/s.  The
    oracle's C calls release the interpreter lock, so the threads run on P
    cores; the oracle itself is unchanged.  All solves start their timed
    blocks together (a barrier after the untimed entry walks); the aggregate
    is the sum of the attempts over the longest thread's time.  Returns
    (rate, P, seconds, walkers sampled per solve)."""
    P = host_cores()
    h, m = _oracle_sample_shape(wl, seconds)
    bar = threading.Barrier(P, timeout=600.0)
    res, err = [None] * P, []

    def work(k):
        try:
            res[k] = _oracle_blocks(wl, h, m, seed + k, seconds, bar)
        except BaseException as e:  # a failed solve breaks the barrier for the others
            bar.abort()
            err.append(e)

    _run_threads(work, P)
    if err:
        raise RuntimeError("oracle timing failed: %r" % (err[0],))
    att = sum(r[0] for r in res)
    el = max(r[1] for r in res)
    return att / el, P, el, h * m


def oracle_time_to_dos(wl, seeds, sweeps, limit_s):
    """The oracle's own time to the converged ln g, seed by seed.  Each
    seed's sweep count is known from the GPU solve (the trajectories are the
    same), so the oracle's time is first estimated from its measured rate;
    if every seed fits in `limit_s`, all seeds are solved by the oracle in
    full, host_cores() at a time in threads, each timed from create to done
    (and its sweep count checked); otherwise the per-seed times are the
    estimate, and the result says so."""
    import concurrent.futures

    rate, _, _, _ = oracle_rate(wl, seeds[0], 3.0)
    per_trial = 1.0 / rate
    est = [sw * wl["h"] * wl["m"] * sites(wl) * per_trial for sw in sweeps]
    out = {"single_core_attempts_per_s": rate, "estimated_s": est}
    if max(est) > limit_s:
        out["measured"] = False
        out["per_seed_s"] = est
        out["how"] = ("estimated, an upper bound: GPU sweep count of each seed x every walker x oracle seconds "
                      "per trial (measured single-threaded; windows that finish early stop costing, which the "
                      "bound ignores); a full oracle solve would exceed %.0f s" % limit_s)
        return out
    from oracle import OracleREWL

    def solve(sd):
        t0 = time.perf_counter()
        O = OracleREWL(wl["model"], wl["L"], wl["h"], OVERLAP, wl["m"], FLATNESS, wl["lnf_final"], sd, q=wl["q"],
                       sweeps_per_exchange=SPE, sweeps_per_flat_check=SPF)
        while not O.run_blocks(SPF // SPE):
            pass
        el = time.perf_counter() - t0
        return el, O.info()["sweep_clock"], O.joined_lng()

    P = min(host_cores(), len(seeds))
    t0 = time.perf_counter()
    with concurrent.futures.ThreadPoolExecutor(max_workers=P) as ex:
        res = list(ex.map(solve, seeds))
    out.update({"measured": True, "threads": P, "wall_s": time.perf_counter() - t0,
                "per_seed_s": [r[0] for r in res], "sweeps": [int(r[1]) for r in res],
                "how": "every seed solved by the oracle in full, %d at a time (one thread each)" % P})
    out["_lng"] = [r[2] for r in res]
    return out


def run_reference(args, wl, world, rank):
    """The reference arm: the plain CPU oracle on the host's cores, as P =
    host_cores() independent solves (one thread each, seeds 0 .. P-1) that
    run their exchange blocks at the same time.  A step is one exchange block
    (100 sweeps) of every solve; the step's time is the slowest solve's."""
    if rank != 0:
        return
    from oracle import OracleREWL

    P = host_cores()
    h, m = _oracle_sample_shape(wl, 2.0)
    per_step = SPE * sites(wl) * h * m
    solves = [OracleREWL(wl["model"], wl["L"], h, OVERLAP, m, FLATNESS, wl["lnf_final"], k, q=wl["q"],
                         sweeps_per_exchange=SPE, sweeps_per_flat_check=SPF) for k in range(P)]

    err = []

    def block(k):
        try:
            solves[k].run_blocks(1)
        except BaseException as e:
            err.append(e)

    def one_step():
        t0 = time.perf_counter()
        _run_threads(block, P)
        if err:
            raise RuntimeError("oracle block failed: %r" % (err[0],))
        return time.perf_counter() - t0

    for _ in range(args.warmup):
        one_step()
    times = [one_step() for _ in range(args.steps)]
    tot = sum(times)
    value = args.steps * P * per_step / tot
    what = ("the %s workload (%d walkers x %d sites)" % (args.workload, h * m, sites(wl)) if h * m == wl["h"] * wl["m"]
            else "the %s lattice with 2 windows x 1 walker (a block of all %d walkers would take minutes)"
            % (args.workload, wl["h"] * wl["m"]))
    sample = ("per step, one block of %d sweeps of %s in each of %d independent oracle solves run at once "
              "(one thread each; seeds 0..%d)" % (SPE, what, P, P - 1))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "attempts/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "desc": wl["desc"],
                       "step": "one exchange block (100 sweeps) of each of %d oracle solves" % P},
            "cpu_baseline": {"value": value, "unit": "attempts/s", "cores": P, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "attempts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gb300(args, wl, world, rank, local):
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    from paper_1305_5615_gb300 import rewl

    rewl.load()
    seed = replica_seed(args.seed, rank)
    stream = torch.cuda.Stream()
    mode = rewl.MODE_GRAPH if args.mode == "graph" else rewl.MODE_PLAIN

    tuned, tune_res = {}, None
    if args.autotune:  # launch shape timed on this problem before the timed region (same bits either way)
        tuned, tune_res = rewl.rewl_autotune(wl["model"], wl["L"], wl["h"], OVERLAP, wl["m"], FLATNESS,
                                             wl["lnf_final"], seed, q=wl["q"], sweeps=2 * SPE,
                                             sweeps_per_exchange=SPE, sweeps_per_flat_check=SPF)

    def make():
        return rewl.REWL(wl["model"], wl["L"], wl["h"], OVERLAP, wl["m"], FLATNESS, wl["lnf_final"], seed, q=wl["q"],
                         sweeps_per_exchange=SPE, sweeps_per_flat_check=SPF, stream=stream, profile=True, mode=mode,
                         **tuned)

    D = make()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        D.step(SPF)
    i0 = dict(D.info)
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xFF)          # L2 flush between timed steps (not inside the events)
        ev[k][0].record(stream)
        D.step(SPF)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    step_ms = [a.elapsed_time(b) for a, b in ev]
    i1 = dict(D.info)
    t_local = sum(step_ms) / 1e3
    att_local = i1["attempts"] - i0["attempts"]
    launches = i1["sweep_launches"] - i0["sweep_launches"]
    sweep_ms = i1["sweep_ms"] - i0["sweep_ms"]
    value, t_max, att_sum = aggregate_replicas(t_local, att_local, world)

    # ---- end to end through the C ABI with host buffers: create (H2D of the
    # problem), one flatness period, the joined ln g read back (D2H), destroy
    e2e_times, h2d, d2h, e2e_att, parts = [], [], [], 0, []
    for k in range(args.e2e_steps):
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xFF)          # same L2 state as the device-timed steps
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        E = make()
        t1 = time.perf_counter()
        E.step(SPF)
        t2 = time.perf_counter()
        g, e0, de = E.lng()
        inf = rewl.rewl_get_info(E._h)   # counters include the ln g read-back
        t3 = time.perf_counter()
        E.close()
        torch.cuda.synchronize()
        t4 = time.perf_counter()
        e2e_times.append(t4 - t0)
        parts.append((t1 - t0, t2 - t1, t3 - t2, t4 - t3))
        h2d.append(inf["h2d_bytes"])
        d2h.append(inf["d2h_bytes"])
        e2e_att += inf["attempts"]
    e2e = None
    if e2e_times:
        e2e = {"value": e2e_att / sum(e2e_times), "unit": "attempts/s",
               "h2d_bytes_per_step": int(statistics.mean(h2d)), "d2h_bytes_per_step": int(statistics.mean(d2h)),
               "step": "rewl_create (H2D of the problem, entry walks) + rewl_step(1000 sweeps: the first flatness "
                       "period of a fresh solve, sweeps 0-1000) + rewl_get_lng (D2H and the host join) + "
                       "rewl_destroy, host buffers, L2 flushed before each step",
               "ms_per_step": {"create": 1e3 * statistics.mean(p[0] for p in parts),
                               "sweeps": 1e3 * statistics.mean(p[1] for p in parts),
                               "read_back": 1e3 * statistics.mean(p[2] for p in parts),
                               "destroy": 1e3 * statistics.mean(p[3] for p in parts)}}

    # ---- roofline of the dominant kernel (the sweep kernel)
    peaks = measured_peaks()
    f_max = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6
    roof = None
    if launches > 0:
        att_per_launch = att_local / launches
        avg_s = sweep_ms / launches / 1e3
        achieved = att_per_launch * OPS_PER_ATTEMPT / avg_s / 1e12
        rate = measured_int_rate()
        peak = N_SM * (rate or 128.0) * f_max / 1e12
        traffic = traffic_from_profile(args.workload, i1["sweep_variant"])
        names = {0: "k_sweep_chain", 1: "k_sweep_spec", 2: "k_sweep_ring"}
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": names.get(i1["sweep_variant"], "k_sweep"), "avg_launch_ms": avg_s * 1e3,
                "attempts_per_launch": att_per_launch, "ops_per_attempt": OPS_PER_ATTEMPT,
                "peak_basis": ("measured: %.1f integer lane-ops/clk/SM (the fastest integer mix of ubench/rates.cu, "
                               "profiles/ubench_pipe_rates_and_wl_step_latency.txt) x 152 SMs x %.0f MHz"
                               % (rate, f_max / 1e6)) if rate else
                              "derived: 152 SMs x 128 int lanes/clk x %.0f MHz (no microbenchmark summary)" % (f_max / 1e6),
                "sweep_share_of_step": sweep_ms / 1e3 / t_local if t_local > 0 else None}
        ph = measured_philox_rate()
        if ph:   # every trial needs one Philox4x32-10 call: a bound of its own
            roof["philox_bound_attempts_per_s"] = ph * N_SM * f_max
            roof["frac_of_philox_bound"] = att_per_launch / avg_s / (ph * N_SM * f_max)
        iso = isolated_step_cycles()
        f_run = (clocks or {}).get("sm_mhz") or f_max / 1e6
        cyc = avg_s * f_run * 1e6 / (SPE * sites(wl))  # per trial of one walker (all walkers run at once)
        if iso is not None:
            walkers = att_per_launch / (SPE * sites(wl))
            roof["latency"] = {"unit": "clk/trial per walker", "kernel": cyc, "isolated_step": iso,
                               "frac": iso / cyc, "sm_mhz": f_run, "walkers": walkers,
                               "chain_bound_attempts_per_s": walkers * f_run * 1e6 / iso,
                               "basis": "the sequential WL step alone (dependency chain only), measured by "
                                        "ubench/rates.cu on the GB300; bound = walkers x SM clock / its cycles"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        rate, blocks, el, n_walk = oracle_rate(wl, seed, args.cpu_seconds)
        what = ("the same workload" if n_walk == wl["h"] * wl["m"] else
                "the same lattice with 2 windows x 1 walker (a block of all %d walkers would take minutes)"
                % (wl["h"] * wl["m"]))
        cpu = {"value": rate, "unit": "attempts/s", "cores": 1, "kind": "oracle",
               "sample": "%d exchange blocks (%d sweeps) of %s, %.1f s, entry walk excluded"
                         % (blocks, blocks * SPE, what, el)}
        if args.cpu_all_cores:
            rate_p, P, el_p, _ = oracle_rate_all_cores(wl, seed, args.cpu_seconds)
            cpu["all_cores"] = {"value": rate_p, "unit": "attempts/s", "cores": P, "kind": "oracle",
                                "sample": "%d independent oracle solves of %s (seeds %d..%d), one thread each, "
                                          "%.1f s of whole exchange blocks at the same time" % (
                                              P, what, seed, seed + P - 1, el_p)}

    tdos = None
    if rank == 0 and world == 1 and args.workload == DEFAULT_WORKLOAD and not args.no_tdos:
        # the metric's second half: time to the converged ln g, served vs plain, p50/p99
        tdos = {"ising-L8-h4-m2": tdos_record(rewl, WORKLOADS["ising-L8-h4-m2"], list(range(32)), _exact_ising(8)),
                "ising-L32-h16-m4": tdos_record(rewl, WORKLOADS["ising-L32-h16-m4"], list(range(8)), _exact_ising(32))}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "attempts/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": args.workload, "desc": wl["desc"], "mode": args.mode,
                           "lanes_per_walker": i1["lanes_per_walker"], "walkers_per_block": i1["walkers_per_block"],
                           "step": "one flatness period: 10 x (100 sweeps + exchange) + flatness/merge",
                           "l2": "flushed between timed steps (256 MiB write, outside the events)",
                           "parallelism": "replicas x%d (independent seeds)" % world,
                           "launch_shape": "autotuned: %s" % json.dumps(
                               [{k: r[k] for k in ("sweep_variant", "lanes_per_walker", "walkers_per_block",
                                                   "ms_per_launch")} for r in tune_res]) if tune_res else
                           "automatic (sweep_variant %d)" % i1["sweep_variant"]},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": args.steps * (3 * (SPF // SPE) + 1), "clocks": clocks,
                "solve_state": {"sweep_clock": i1["sweep_clock"], "windows_done": i1["windows_done"]},
                "time_to_dos": tdos}
        print(json.dumps(line), flush=True)


SERVED_MIX = (("ea", (12, 16, 20, 24, 32), 2), ("ising", (16, 24, 32), 2), ("potts", (16, 24, 32), 10))


def served_requests(n, seed):
    """The served stream: model uniform over {+-J, Ising, Potts q=10} (1/3 each),
    L uniform over the model's sizes, 8 windows at 75% overlap x 4 walkers,
    flatness 0.8, ln f -> 1e-6, request seed = request index (+-J couplings
    drawn from it with p = 1/2)."""
    import numpy as np

    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        model, sizes, q = SERVED_MIX[int(rng.integers(3))]
        out.append(dict(model=model, L=int(sizes[int(rng.integers(len(sizes)))]), q=q, seed=i))
    return out


def _fifo_latencies(arrivals, services):
    """One server, first come first served: latency of each job (Lindley)."""
    free_at, lat = 0.0, []
    for a, sv in zip(arrivals, services):
        start = max(a, free_at)
        free_at = start + sv
        lat.append(free_at - a)
    return lat


def _plain_request(rewl, r, stop=None):
    """One request solved in plain form on its own handle (and stream):
    rewl_create + rewl_step to completion + rewl_get_lng, in steps of one
    flatness period, abandoned when `stop` (a threading.Event) is set.
    Returns (ln g or None if abandoned, attempts)."""
    D = rewl.REWL(r["model"], r["L"], 8, OVERLAP, 4, FLATNESS, 1e-6, r["seed"], q=r["q"])
    done = False
    while not done and not (stop is not None and stop.is_set()):
        done = D.step(SPF)
    g = D.lng()[0] if done else None
    att = int(D.info["attempts"])
    D.close()
    return g, att


def run_plain_stream(rewl, reqs, arrivals, concurrency, stop_after=0.0):
    """The plain form over a stream: every request is solved by its own
    rewl_create/rewl_step handle on its own stream, started at its arrival by
    a host thread, at most `concurrency` at once (first come first served
    beyond that); with stop_after > 0 the requests still running after that
    many seconds are abandoned.  Returns per-request latency (arrival ->
    result; None if unfinished), (ln g, attempts) per request, and the wall
    time."""
    n = len(reqs)
    sem = threading.Semaphore(concurrency)
    stop = threading.Event()
    lat, res = [None] * n, [(None, 0)] * n
    err = []
    t0 = time.perf_counter()

    def run(k):
        try:
            with sem:
                if stop.is_set():
                    return
                res[k] = _plain_request(rewl, reqs[k], stop)
            if res[k][0] is not None:
                lat[k] = time.perf_counter() - t0 - arrivals[k]
        except BaseException as e:
            err.append(e)

    threads = []
    for k in range(n):
        delay = arrivals[k] - (time.perf_counter() - t0)
        if stop_after > 0:
            delay = min(delay, stop_after - (time.perf_counter() - t0))
        if delay > 0:
            time.sleep(delay)
        if stop_after > 0 and time.perf_counter() - t0 >= stop_after:
            break
        th = threading.Thread(target=run, args=(k,))
        th.start()
        threads.append(th)
    if stop_after > 0:
        while any(th.is_alive() for th in threads) and time.perf_counter() - t0 < stop_after:
            time.sleep(0.05)
        stop.set()
    for th in threads:
        th.join()
    if err:
        raise RuntimeError("plain solve failed: %r" % (err[0],))
    return lat, res, min(time.perf_counter() - t0, stop_after) if stop_after > 0 else time.perf_counter() - t0


def run_served_stream(rewl, reqs, arrivals, slots, server_gb, timeout_s):
    """The served form over a stream: each request submitted at its arrival
    to one request server (continuous batching); stops after timeout_s
    seconds (> 0).  Returns per-request latency (arrival -> result; None if
    unfinished), (ln g, attempts) per request, wall time and the server's
    rounds."""
    S = rewl.RewlServer(device_bytes=server_gb << 30, max_running=slots)
    ids, t_sub = [], []
    t0 = time.perf_counter()
    nxt = 0
    st = {"rounds": 0}
    while True:
        now = time.perf_counter() - t0
        while nxt < len(reqs) and arrivals[nxt] <= now:
            r = reqs[nxt]
            ids.append(S.submit(r["model"], r["L"], 8, OVERLAP, 4, FLATNESS, 1e-6, r["seed"], q=r["q"]))
            t_sub.append(time.perf_counter() - t0)
            nxt += 1
        st = S.run(1)
        if nxt == len(reqs) and st["running"] == 0 and st["queued"] == 0:
            break
        if timeout_s > 0 and time.perf_counter() - t0 > timeout_s:
            break
        if st["running"] == 0 and st["queued"] == 0 and nxt < len(reqs):
            time.sleep(max(0.0, arrivals[nxt] - (time.perf_counter() - t0)))
    wall = time.perf_counter() - t0
    lat, res = [], []
    for k, rid in enumerate(ids):
        inf = S.poll(rid)
        if inf["state"] == rewl.REQ_DONE:
            lat.append(t_sub[k] - arrivals[k] + inf["latency_ms"] / 1e3)
            res.append((S.result(rid)[0], int(inf["attempts"])))
        else:
            lat.append(None)
            res.append((None, int(inf["attempts"])))
    lat += [None] * (len(reqs) - len(ids))
    res += [(None, 0)] * (len(reqs) - len(ids))
    S.close()
    return lat, res, wall, st["rounds"]


def _summary(lat, res, wall):
    import numpy as np

    done = [x for x in lat if x is not None]
    att = sum(r[1] for r in res)
    return {"completed": len(done), "unfinished": len(lat) - len(done), "wall_s": wall,
            "attempts_per_s": att / wall, "completed_per_s": len(done) / wall,
            "p50_latency_s": float(np.percentile(done, 50)) if done else None,
            "p99_latency_s": float(np.percentile(done, 99)) if done else None}


def run_served(args, world, rank, local):
    """A stream of DOS requests, served form against plain form, both measured.

    Plain form: every request solved by its own handle (one launch per phase,
    its own stream), up to --slots at once.  Calibration (--rate < 0): a
    backlog of --calib-requests requests of the mix through the plain form for
    --calib-seconds gives its capacity C (requests completed per second); the
    stream then arrives as a Poisson process at rate lambda = -rate x C (0.8 x C
    for --rate -0.8) for --arrival-window seconds.  The same arrivals go
    through the request server (served) and through the plain form, each arm
    stopped --drain seconds after the last arrival; p50/p99 latency from
    arrival to result over the requests each arm finished and over those both
    finished, aggregate attempts/s, and the ln g of every request both finished
    compared bit for bit."""
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    from paper_1305_5615_gb300 import rewl

    rewl.load()
    calib = None
    rate = args.rate
    if rate < 0:
        creq = served_requests(args.calib_requests, args.seed + 1000)
        for i, r in enumerate(creq):
            r["seed"] = 100000 + i
        clat, cres, cwall = run_plain_stream(rewl, creq, [0.0] * len(creq), args.slots, args.calib_seconds)
        done = sum(1 for x in clat if x is not None)
        cap = max(done, 1) / cwall
        rate = -args.rate * cap
        calib = {"requests": len(creq), "concurrency": args.slots, "seconds": cwall, "completed": done,
                 "plain_capacity_requests_per_s": cap, "load_factor": -args.rate, "rate_per_s": rate}
        print("calibration: %s" % json.dumps(calib), file=sys.stderr, flush=True)
    rng = np.random.default_rng(args.seed + 1)
    if rate > 0:
        arrivals = list(np.cumsum(rng.exponential(1.0 / rate, size=100000)))
        arrivals = [a for a in arrivals if a < args.arrival_window][:args.requests]
    else:
        arrivals = [0.0] * args.requests
    reqs = served_requests(len(arrivals), args.seed)
    if args.mix != "mixed":  # one shape only, e.g. "ising:32"
        model, L = args.mix.split(":")
        reqs = [dict(model=model, L=int(L), q=10 if model == "potts" else 2, seed=i) for i in range(len(reqs))]
    horizon = (arrivals[-1] if arrivals else 0.0) + args.drain
    slat, sres, swall, srounds = run_served_stream(rewl, reqs, arrivals, args.slots, args.server_gb, horizon)
    served = _summary(slat, sres, swall)
    served["rounds"] = srounds
    print("served: %s" % json.dumps(served), file=sys.stderr, flush=True)
    plain, same, both = None, None, None
    if not args.no_plain:
        plat, pres, pwall = run_plain_stream(rewl, reqs, arrivals, args.slots, horizon)
        plain = _summary(plat, pres, pwall)
        print("plain: %s" % json.dumps(plain), file=sys.stderr, flush=True)
        idx = [k for k in range(len(reqs)) if slat[k] is not None and plat[k] is not None]
        same = all(np.array_equal(sres[k][0].view(np.uint64), pres[k][0].view(np.uint64)) for k in idx)
        if idx:
            both = {"requests": len(idx),
                    "served_p50_s": float(np.percentile([slat[k] for k in idx], 50)),
                    "served_p99_s": float(np.percentile([slat[k] for k in idx], 99)),
                    "plain_p50_s": float(np.percentile([plat[k] for k in idx], 50)),
                    "plain_p99_s": float(np.percentile([plat[k] for k in idx], 99))}
    if rank == 0:
        print(json.dumps({"metric": "served DOS requests: p50/p99 arrival->result and aggregate spin-flip attempts/s, "
                                    "served vs plain",
                          "value": served["attempts_per_s"], "unit": "attempts/s", "n_gpus": world,
                          "higher_is_better": True, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": "served-stream", "requests": len(reqs),
                                     "desc": "+-J L in {12,16,20,24,32} (p=1/2 couplings from the request seed), "
                                             "Ising and Potts q=10 L in {16,24,32}, 1/3 each; 8 windows x 4 walkers; "
                                             "ln f -> 1e-6; arrivals %s; each arm stopped %.0f s after the last "
                                             "arrival" % ("Poisson %.4g/s over %.0f s" % (rate, args.arrival_window)
                                                          if rate > 0 else "all at t=0 (backlog)", args.drain),
                                     "slots": args.slots, "plain": "one handle per request on its own stream, up to "
                                                                   "%d at once" % args.slots},
                          "calibration": calib, "served": served, "plain": plain,
                          "finished_by_both": both, "results_bit_identical_served_vs_plain": same}), flush=True)


def _first_iteration(rewl, wl, seed, max_sweeps, **kw):
    """Runs a solve until every window has finished its first iteration (or the
    sweep budget ends); returns (state, info, seconds)."""
    D = rewl.REWL(wl["model"], wl["L"], wl["h"], OVERLAP, wl["m"], FLATNESS, wl["lnf_final"], seed, q=wl["q"], **kw)
    t0 = time.perf_counter()
    while True:
        D.step(SPF)
        st = D.state()
        if (st["first_iter"] > 0).all() or st["sweep_clock"] >= max_sweeps:
            break
    el = time.perf_counter() - t0
    info = dict(D.info)
    D.close()
    return st, info, el


def run_windows_balance(args, world, rank, local):
    """Fig. 1b against Fig. 1a: sweeps until every window has finished its
    first WL iteration (the paper's speed-up counts the sweeps of the slowest
    walker, Eq. (2)), with equal windows and with the run-time balanced
    partition planned from that equal run (rewl_plan_windows)."""
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    from paper_1305_5615_gb300 import rewl

    wl = WORKLOADS[args.base_workload]
    eq, info_eq, t_eq = _first_iteration(rewl, wl, args.seed, args.max_sweeps)
    starts, widths = rewl.rewl_plan_windows(eq["first_iter"], eq["win_start"], eq["win_width"], info_eq["n_bins"],
                                            wl["h"], OVERLAP)
    out = {"equal": None, "balanced": None}
    for name, st, el, ww in (("equal", eq, t_eq, eq["win_width"]),):
        fi = st["first_iter"]
        out[name] = {"slowest_window_sweeps": int(fi.max()), "fastest_window_sweeps": int(fi[fi > 0].min()),
                     "first_iter_sweeps": [int(x) for x in fi], "widths": [int(x) for x in ww], "seconds": el}
    seeds = [args.seed + k for k in range(args.balance_seeds)]
    runs = []
    for sd in seeds:
        b, info_b, t_b = _first_iteration(rewl, wl, sd, args.max_sweeps, window_starts=starts, window_widths=widths)
        e, info_e, t_e = (eq, info_eq, t_eq) if sd == args.seed else _first_iteration(rewl, wl, sd, args.max_sweeps)
        runs.append((int(e["first_iter"].max()), int(b["first_iter"].max())))
        if sd == args.seed:
            fi = b["first_iter"]
            out["balanced"] = {"slowest_window_sweeps": int(fi.max()), "fastest_window_sweeps": int(fi[fi > 0].min()),
                               "first_iter_sweeps": [int(x) for x in fi], "starts": [int(x) for x in starts],
                               "widths": [int(x) for x in widths], "seconds": t_b}
    ratio = float(np.mean([e / b for e, b in runs]))
    if rank == 0:
        print(json.dumps({"metric": "sweeps until every window finished its first WL iteration (slowest window), "
                                    "equal vs run-time balanced windows",
                          "value": ratio, "unit": "speed-up (equal / balanced)", "n_gpus": world,
                          "higher_is_better": True, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": "windows-balance", "base": args.base_workload, "desc": wl["desc"],
                                     "seeds": seeds, "plan_from_seed": args.seed},
                          "per_seed_slowest_sweeps_equal_balanced": runs, "detail": out}), flush=True)


def _exact_ising(L):
    """ln g of the exact L x L Ising DOS (tests/golden, written from the
    Kaufman/Beale closed form), indexed by global bin (E = -2N + 4 b); -inf
    for levels that do not exist."""
    import math

    import numpy as np

    N = L * L
    out = np.full(N + 1, -np.inf)
    for line in open(os.path.join(ROOT, "tests", "golden", "ising_L%d_exact_dos.txt" % L)):
        if line.startswith("#"):
            continue
        e, c = line.split()
        c = int(c)
        if c == 0:
            continue
        b = c.bit_length()
        out[(int(e) + 2 * N) // 4] = math.log(c) if b < 1000 else math.log(c >> (b - 60)) + (b - 60) * math.log(2.0)
    return out


def _exact_ising_L32():
    return _exact_ising(32)


def dos_accuracy(g, e0, de, lnx):
    """Max relative error |ln g - ln g_exact| / ln g_exact of each half of the
    estimate normalised at its own end (E <= 0 with g(E_min) = 2, E >= 0 with
    g(E_max) = 2), and the max absolute deviation after the best shift."""
    import numpy as np

    fin = np.isfinite(lnx)
    E = e0 + de * np.arange(len(g))
    lo, hi = fin & (E <= 0), fin & (E >= 0)
    top = np.nonzero(fin)[0][-1]
    g_lo, g_hi = g - g[0] + lnx[0], g - g[top] + lnx[top]
    d = g[fin] - lnx[fin]
    return {"max_rel_err_E_le_0": float(np.max(np.abs(g_lo[lo] - lnx[lo]) / lnx[lo])),
            "max_rel_err_E_ge_0": float(np.max(np.abs(g_hi[hi] - lnx[hi]) / lnx[hi])),
            "max_abs_err_best_shift": float(np.max(np.abs(d - d.mean())))}


def tdos_record(rewl, wl, seeds, exact=None, alone=True):
    """Time to the converged ln g (every window at ln f_final), measured three
    ways on the same seeds, each from submission / creation to the result:
      served  -- all seeds submitted at once to the request server (continuous
                 batching: one fused launch per phase for all requests);
      plain, concurrent -- one rewl_create + rewl_step(to completion) +
                 rewl_get_lng handle per seed, each on its own stream driven by
                 its own host thread, all started together (one launch per
                 phase per solve);
      plain, alone -- the first seed solved by itself on the GPU.
    p50/p99 over the seeds, the served results checked bit for bit against the
    plain ones, and (exact DOS given) each seed's error against it."""
    import numpy as np

    rec = {"seeds": list(seeds), "lnf_final": wl["lnf_final"]}
    # ---- served
    S = rewl.RewlServer(device_bytes=8 << 30, max_running=len(seeds))
    t0 = time.perf_counter()
    ids = [S.submit(wl["model"], wl["L"], wl["h"], OVERLAP, wl["m"], FLATNESS, wl["lnf_final"], sd, q=wl["q"])
           for sd in seeds]
    while True:
        st = S.run(1)
        if st["running"] == 0 and st["queued"] == 0:
            break
    wall = time.perf_counter() - t0
    lat, sweeps, served_g = [], [], []
    for rid in ids:
        inf = S.poll(rid)
        assert inf["state"] == rewl.REQ_DONE, inf
        lat.append(inf["latency_ms"] / 1e3)
        sweeps.append(int(inf["sweeps"]))
        served_g.append(S.result(rid))
    rec["served"] = {"wall_s": wall, "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                     "per_seed_s": lat, "attempts_per_s": st["attempts"] / wall}
    rec["sweeps_to_converge"] = sweeps
    S.close()

    # ---- plain, concurrent
    res = [None] * len(seeds)
    start = threading.Barrier(len(seeds), timeout=600.0)

    def solve(k):
        start.wait()
        t1 = time.perf_counter()
        D = rewl.REWL(wl["model"], wl["L"], wl["h"], OVERLAP, wl["m"], FLATNESS, wl["lnf_final"], seeds[k], q=wl["q"])
        D.step(0)
        g = D.lng()
        res[k] = (time.perf_counter() - t1, g, int(D.info["attempts"]), int(D.info["sweep_clock"]))
        D.close()

    t0 = time.perf_counter()
    _run_threads(solve, len(seeds))
    wall = time.perf_counter() - t0
    pl = [r[0] for r in res]
    rec["plain_concurrent"] = {"wall_s": wall, "p50_s": float(np.percentile(pl, 50)),
                               "p99_s": float(np.percentile(pl, 99)), "per_seed_s": pl,
                               "attempts_per_s": sum(r[2] for r in res) / wall}
    rec["bit_identical_served_vs_plain"] = all(
        np.array_equal(r[1][0].view(np.uint64), g[0].view(np.uint64)) for r, g in zip(res, served_g))
    rec["sweeps_equal_served_vs_plain"] = [r[3] for r in res] == sweeps
    # ---- plain, alone
    if alone:
        t1 = time.perf_counter()
        D = rewl.REWL(wl["model"], wl["L"], wl["h"], OVERLAP, wl["m"], FLATNESS, wl["lnf_final"], seeds[0], q=wl["q"])
        D.step(0)
        D.lng()
        rec["plain_alone"] = {"seed": seeds[0], "s": time.perf_counter() - t1,
                              "attempts_per_s": D.info["attempts"] / (time.perf_counter() - t1)}
        D.close()
    if exact is not None:
        acc = [dos_accuracy(g, e0, de, exact) for g, e0, de in served_g]
        rec["accuracy_vs_exact"] = {
            "per_seed": acc,
            "worst_max_rel_err_E_le_0": max(a["max_rel_err_E_le_0"] for a in acc),
            "worst_max_rel_err_E_ge_0": max(a["max_rel_err_E_ge_0"] for a in acc),
            "seeds_within_2e-3": sum(1 for a in acc if max(a["max_rel_err_E_le_0"], a["max_rel_err_E_ge_0"]) <= 2e-3),
            "mean_of_seeds": dos_accuracy(np.mean([g for g, _, _ in served_g], axis=0), served_g[0][1],
                                          served_g[0][2], exact)}
    return rec


def run_rule_compare(args, world, rank, local):
    """The two WL rules on the GPU (Ising 32 x 32, 16 windows x 4 walkers): for
    each final ln f, the sweeps and seconds to converge and the error against
    the exact DOS (max relative error of ln g over E <= 0 with g(E_min) = 2,
    and the max absolute error after the best constant shift)."""
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    from paper_1305_5615_gb300 import rewl

    ex = _exact_ising_L32()
    fin = np.isfinite(ex)
    half = fin & (-2048 + 4 * np.arange(1025) <= 0)
    res = []
    for rule in ("flat", "1/t"):
        for k in args.rule_k:
            D = rewl.REWL("ising", 32, 16, OVERLAP, 4, FLATNESS, 2.0 ** -k * 0.75, args.seed, wl_rule=rule)
            t0 = time.perf_counter()
            D.step(0)
            el = time.perf_counter() - t0
            g, _, _ = D.lng()
            gn = g - g[0] + ex[0]
            rel = float(np.max(np.abs(gn[half] - ex[half]) / ex[half]))
            d = g[fin] - ex[fin]
            absd = float(np.max(np.abs(d - d.mean())))
            res.append({"rule": rule, "final_lnf": 2.0 ** -k, "sweeps": int(D.info["sweep_clock"]), "seconds": el,
                        "max_rel_err_E_le_0": rel, "max_abs_err_shifted": absd})
            D.close()
    if rank == 0:
        print(json.dumps({"metric": "error against the exact DOS and time to converge, flatness rule vs 1/t rule",
                          "value": None, "unit": None, "n_gpus": world, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": "rule-compare", "desc": WORKLOADS[DEFAULT_WORKLOAD]["desc"],
                                     "seed": args.seed}, "runs": res}), flush=True)


def run_time_to_dos(args, world, rank, local):
    """Time to the converged ln g (every window at ln f_final) over seeds, the
    served form against the plain form.  Served: all seeds submitted at once
    to the request server (their walkers share the GPU); plain: the first
    --tdos-plain seeds solved one after another with rewl_create/rewl_step,
    the others modelled as their own sweep count (identical in both forms)
    times the plain seconds per sweep measured on the solved ones, queued one
    after another.  Reports p50/p99 of both and the result bits of the plain
    solves against the served ones."""
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    from paper_1305_5615_gb300 import rewl

    wl = WORKLOADS[args.base_workload]
    seeds = list(range(args.seed, args.seed + args.tdos_seeds))
    S = rewl.RewlServer(device_bytes=args.server_gb << 30, max_running=len(seeds))
    t0 = time.perf_counter()
    ids = [S.submit(wl["model"], wl["L"], wl["h"], OVERLAP, wl["m"], FLATNESS, wl["lnf_final"], sd, q=wl["q"])
           for sd in seeds]
    while True:
        st = S.run(1)
        if st["running"] == 0 and st["queued"] == 0:
            break
    t_served = time.perf_counter() - t0
    served, sweeps = [], []
    for rid in ids:
        inf = S.poll(rid)
        served.append(inf["latency_ms"] / 1e3)
        sweeps.append(inf["sweeps"])
    tuned, tune_res = {}, None
    if args.autotune:
        tuned, tune_res = rewl.rewl_autotune(wl["model"], wl["L"], wl["h"], OVERLAP, wl["m"], FLATNESS,
                                             wl["lnf_final"], args.seed, q=wl["q"], sweeps=SPF)
    plain, per_sweep, bits, secondary = [], [], [], None
    for k, sd in enumerate(seeds[:args.tdos_plain]):
        t1 = time.perf_counter()
        D = rewl.REWL(wl["model"], wl["L"], wl["h"], OVERLAP, wl["m"], FLATNESS, wl["lnf_final"], sd, q=wl["q"],
                      mode=rewl.MODE_GRAPH if args.mode == "graph" else rewl.MODE_PLAIN, **tuned)
        D.step(0)
        g, _, _ = D.lng()
        el = time.perf_counter() - t1
        plain.append(el)
        per_sweep.append(el / D.info["sweep_clock"])
        bits.append(bool(np.array_equal(g.view(np.uint64), S.result(ids[k])[0].view(np.uint64))))
        if k == 0:
            ds = D.state()
            tried = ds["x_tried"][:-1].astype(np.float64)
            secondary = {"seed": sd, "sweeps_to_converge": int(ds["sweep_clock"]),
                         "iterations_per_window": [int(x) for x in ds["iteration"]],
                         "exchange_acceptance_per_pair": [float(a) / t if t else None for a, t in
                                                          zip(ds["x_accepted"][:-1].astype(np.float64), tried)],
                         "exchange_rounds": int(ds["exchange_rounds"]),
                         "replica_round_trips": int(ds["rep_trips"].sum()),
                         "wl_acceptance": float(ds["wl_accept"].sum()) / float(D.info["attempts"])}
        D.close()
    sps = float(np.mean(per_sweep)) if per_sweep else None
    svc = [plain[k] if k < len(plain) else sps * sweeps[k] for k in range(len(seeds))]
    queued = list(np.cumsum(svc))          # all submitted at t = 0, solved one after another
    orc = None
    if rank == 0 and not args.no_cpu:
        orc = oracle_time_to_dos(wl, seeds, sweeps, args.tdos_oracle_limit)
        lngs = orc.pop("_lng", None)
        if lngs is not None:
            dev = []
            for k, g_o in enumerate(lngs):
                g_s = S.result(ids[k])[0]
                fin = np.isfinite(g_o)
                same_support = bool(np.array_equal(np.isfinite(g_s), fin))
                dev.append(float(np.abs(g_s[fin] - g_o[fin]).max()) if same_support else None)
            orc["sweeps_equal_gpu"] = orc["sweeps"] == [int(s) for s in sweeps]
            orc["max_abs_lng_diff_vs_gpu"] = dev
        orc["p50_s"] = float(np.percentile(orc["per_seed_s"], 50))
        orc["p99_s"] = float(np.percentile(orc["per_seed_s"], 99))
        orc["queued_one_core_p50_s"] = float(np.percentile(np.cumsum(orc["per_seed_s"]), 50))
        orc["queued_one_core_p99_s"] = float(np.percentile(np.cumsum(orc["per_seed_s"]), 99))
    if rank == 0:
        print(json.dumps({"metric": "time to converged ln g (ln f_final), p50/p99 over seeds, served vs plain",
                          "value": float(np.percentile(served, 50)), "unit": "s (served p50)", "n_gpus": world,
                          "higher_is_better": False, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": "time-to-dos", "base": args.base_workload, "desc": wl["desc"],
                                     "seeds": seeds, "plain_mode": args.mode,
                                     "plain_launch_shape": ("autotuned: %s" % json.dumps(
                                         [{k: r[k] for k in ("sweep_variant", "lanes_per_walker", "ms_per_launch")}
                                          for r in tune_res]) if tune_res else "automatic")},
                          "served": {"wall_s": t_served, "p50_s": float(np.percentile(served, 50)),
                                     "p99_s": float(np.percentile(served, 99)), "per_seed_s": served,
                                     "sweeps": sweeps, "attempts_per_s": st["attempts"] / t_served},
                          "plain": {"solved": len(plain), "solved_s": plain, "seconds_per_sweep": sps,
                                    "service_p50_s": float(np.percentile(svc, 50)),
                                    "service_p99_s": float(np.percentile(svc, 99)),
                                    "queued_p50_s": float(np.percentile(queued, 50)),
                                    "queued_p99_s": float(np.percentile(queued, 99)),
                                    "bit_identical_to_served": bits},
                          "secondary": secondary, "oracle": orc}), flush=True)


def run_glass_e0(args, world, rank, local):
    """The 12^3 +-J glass: lowest energy per spin the REWL walk has visited
    after a fixed time, over disorder realisations (seeds), beside the
    paper's e_0 = -1.787 +- 0.005.  The zero-temperature descent that lays out
    the windows is reported too: the walk can go below it (the lowest window
    reaches on to -3N)."""
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    from paper_1305_5615_gb300 import rewl

    wl = WORKLOADS["ea3d-L12-h16-m4"]
    out = []
    for sd in range(args.seed, args.seed + args.glass_samples):
        D = rewl.REWL("ea3d", 12, wl["h"], OVERLAP, wl["m"], FLATNESS, wl["lnf_final"], sd)
        info = D.info
        st0 = D.state()
        e_desc = int(st0["E"].min())
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < args.glass_seconds:
            if D.step(SPF):
                break
        el = time.perf_counter() - t0
        st = D.state()
        lng0 = st["lng"][:wl["m"]]                       # the lowest window's walkers
        visited = np.nonzero((lng0 > 0).any(0))[0]
        e_low = info["e_min"] + 4 * int(visited.min())
        out.append({"seed": sd, "e_desc_per_spin": e_desc / 1728.0, "e_low_per_spin": e_low / 1728.0,
                    "sweeps": int(st["sweep_clock"]), "seconds": el,
                    "round_trips": int(st["rep_trips"].sum()), "replicas": int(len(st["rep_trips"])),
                    "attempts_per_s": rewl.rewl_get_info(D._h)["attempts"] / el})
        D.close()
    lows = np.array([o["e_low_per_spin"] for o in out])
    if rank == 0:
        print(json.dumps({"metric": "lowest energy per spin visited by the REWL walk, 12^3 +-J glass, over seeds",
                          "value": float(lows.mean()), "unit": "e_0 estimate (mean over samples)",
                          "stderr": float(lows.std(ddof=1) / np.sqrt(len(lows))) if len(lows) > 1 else None,
                          "paper_e0": "-1.787 +- 0.005", "n_gpus": world, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": "glass-e0", "desc": wl["desc"], "seconds_per_sample": args.glass_seconds},
                          "samples": out}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS) + ["served-stream", "windows-balance", "rule-compare",
                                                                        "time-to-dos", "glass-e0"])
    ap.add_argument("--mode", default="plain", choices=["plain", "graph"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tdos", action="store_true",
                    help="skip the time-to-DOS records (served vs plain) of the default workload")
    ap.add_argument("--cpu-all-cores", type=int, default=1,
                    help="also time one oracle solve per host core at the same time (0 = single core only)")
    ap.add_argument("--tdos-oracle-limit", type=float, default=300.0,
                    help="time-to-dos: solve the seeds with the oracle in full if each takes less than this (s)")
    ap.add_argument("--autotune", action="store_true", help="time the sweep launch shapes first (rewl_autotune)")
    ap.add_argument("--requests", type=int, default=1000, help="served-stream: at most this many requests")
    ap.add_argument("--rate", type=float, default=-0.8,
                    help="served-stream: Poisson arrivals per second; 0 = all at once; < 0: -rate x the plain "
                         "form's capacity measured in a calibration run first")
    ap.add_argument("--calib-requests", type=int, default=32, help="served-stream: calibration backlog")
    ap.add_argument("--calib-seconds", type=float, default=150.0, help="served-stream: calibration window")
    ap.add_argument("--arrival-window", type=float, default=240.0, help="served-stream: seconds of arrivals")
    ap.add_argument("--drain", type=float, default=240.0,
                    help="served-stream: each arm stops this many seconds after the last arrival")
    ap.add_argument("--no-plain", action="store_true", help="served-stream: skip the plain arm")
    ap.add_argument("--slots", type=int, default=256, help="served-stream: request slots (served) and the "
                                                          "plain form's concurrent handles")
    ap.add_argument("--server-gb", type=int, default=64, help="served-stream: device-memory budget in GiB")
    ap.add_argument("--mix", default="mixed", help="served-stream: 'mixed', or one shape as model:L (e.g. ising:32)")
    ap.add_argument("--served-timeout", type=float, default=1200.0, help="served-stream: stop after this many seconds")
    ap.add_argument("--base-workload", default="potts-q10-L32-h32-m16", choices=sorted(WORKLOADS),
                    help="windows-balance, time-to-dos: the problem")
    ap.add_argument("--balance-seeds", type=int, default=3, help="windows-balance: seeds compared")
    ap.add_argument("--max-sweeps", type=int, default=2000000, help="windows-balance: sweep budget per run")
    ap.add_argument("--rule-k", type=int, nargs="+", default=[16, 20], help="rule-compare: final ln f = 2^-k")
    ap.add_argument("--tdos-seeds", type=int, default=8, help="time-to-dos: seeds")
    ap.add_argument("--tdos-plain", type=int, default=1, help="time-to-dos: seeds also solved plain in full")
    ap.add_argument("--glass-samples", type=int, default=4, help="glass-e0: disorder realisations")
    ap.add_argument("--glass-seconds", type=float, default=60.0, help="glass-e0: walk time per realisation")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world, rank, local = dist_setup()
    if args.workload == "served-stream":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the served stream has no CPU reference arm"}))
            return
        run_served(args, world, rank, local)
        return
    if args.workload == "glass-e0":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the glass e_0 run has no CPU reference arm"}))
            return
        run_glass_e0(args, world, rank, local)
        return
    if args.workload == "time-to-dos":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "time-to-DOS over seeds has no CPU reference arm"}))
            return
        run_time_to_dos(args, world, rank, local)
        return
    if args.workload == "rule-compare":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the rule comparison has no CPU reference arm"}))
            return
        run_rule_compare(args, world, rank, local)
        return
    if args.workload == "windows-balance":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the window-balance comparison has no CPU reference arm"}))
            return
        run_windows_balance(args, world, rank, local)
        return
    wl = WORKLOADS[args.workload]
    if world > 1 and args.impl == "gb300":
        import torch.distributed as dist
        import torch

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    if args.impl == "reference":
        run_reference(args, wl, world, rank)
    else:
        run_gb300(args, wl, world, rank, local)
    if world > 1 and args.impl == "gb300":
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
