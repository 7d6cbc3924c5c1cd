"""Benchmark of the per-step stress-transfer functional on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload six_fault_3072]

Workload: the six-fault, 3072-element network run for its full 2000 steps, with the selective H-matrix (leaf 32,
eta_H 2, ACA 1e-6) and the causal / spectral windows.  A step is one push of the slip rate plus one seas_stress_step
(all hot-path stages: push, forward FFT, mode convolution, H-matrix interaction and its reduction, inverse FFT +
assembly).  The operator is always built for the 2000-step workload; each scenario is advanced untimed to step
2000 - K (the last W of those steps are the warm-up) and the K deepest steps, [2000 - K, 2000), are timed, so the
timed steps carry the full history depth whatever K is.  Prints one JSON line.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

if "--impl" in sys.argv and "reference" in sys.argv:      # the oracle arm runs single-threaded per process
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(var, "1")

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2603_00383_gb300 import synth  # noqa: E402

METRIC = "element-steps/s"
# name -> (seas precision code, dtype label of the arithmetic)
PRECISIONS = {"fp64": (0, "f64"), "df64": (3, "df64 (fp32 pairs)"), "bf16": (1, "bf16 storage, f32 compensated"),
              "fp16s": (2, "fp16 storage with per-slice scale, f32 compensated")}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200, help="timed steps K: the K deepest steps of the workload")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="six_fault_3072")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 dense comparison run")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-sample", type=int, default=48, help="oracle element-steps in the CPU baseline")
    ap.add_argument("--precision", default="fp64", choices=list(PRECISIONS), help="headline storage precision")
    ap.add_argument("--no-variants", action="store_true", help="skip the other storage precisions")
    ap.add_argument("--no-batched", action="store_true", help="skip the 8-scenario ensemble runs")
    ap.add_argument("--no-tail", action="store_true", help="skip the static-tail run")
    ap.add_argument("--no-cluster", action="store_true", help="skip the cluster-level end truncation run")
    ap.add_argument("--no-surface", action="store_true", help="skip the free-surface (method of images) run")
    ap.add_argument("--no-oracle-rows", action="store_true", help="skip the oracle interaction rows (errors)")
    ap.add_argument("--dump-step-bytes", default=None, help="write the per-step algorithmic interaction bytes here")
    ap.add_argument("--served-seconds", type=float, default=15.0, help="wall time of the served run (0: skip)")
    ap.add_argument("--max-steps", type=int, default=None,
                    help="build the workload for this many steps instead (smaller operators for profiling captures)")
    ap.add_argument("--batched-only", action="store_true", help="only the 8-scenario ensemble runs (profiling)")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the 8 geometries x 8 scenarios run")
    return ap.parse_args()


def log(msg):
    print(f"[bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def window(w, K):
    """The timed window [start, steps): the K deepest steps of the workload."""
    K = max(1, min(int(K), w.steps))
    return w.steps - K, K


# ------------------------------------------------------------------------------------------------ oracle sample --

def oracle_sample(w, start, K, count, seed=11):
    """(element, step) pairs of the CPU-baseline / reference sample: elements of fault 0 (whose spectral tables the
    oracle builds once, untimed), steps spread over the timed window."""
    n0 = int(w.faults[0, 4])
    k = np.arange(count)
    elems = (k * 97 + seed) % n0
    steps = start + (k * 7919 + 13 * seed) % K
    return elems, steps


def oracle_rows(w):
    """Receivers of the interaction-error check: two per fault (first and middle element)."""
    off = np.concatenate([[0], np.cumsum(w.faults[:, 4].astype(int))])
    return np.array([r for f in range(w.n_faults) for r in (off[f], (off[f] + off[f + 1]) // 2)])


class OracleStepper:
    """Evaluates tau at single (element, step) pairs with the CPU oracle (interaction row + spectral self term of
    fault 0 + radiation damping), with the workload's windows."""

    def __init__(self, w, tables=None):
        from oracle import seas_oracle as O
        self.O = O
        self.w = w
        self.net = O.network(w.faults, w.mu, w.cs)
        hp = w.hparams
        self.V = w.slip_rate(0, 0, w.steps)
        self.delta = O.slip_from_rate(self.V, self.net.dt)
        no_trunc = bool(hp.get("flags", 0) & 2)
        _, _, self.last = O.pair_windows(self.net, hp["eta_tmin"], hp["eta_tmax"], hp["max_steps"], no_trunc)
        n0 = int(self.net.n_elem[0])
        if tables is None:
            W0 = O.mode_windows(n0, self.net.length[0], self.net.dt, self.net.cs, hp["eta_w"], hp["q_w"],
                                hp["max_steps"], no_trunc)
            tables = O.SelfTables(n0, self.net.length[0], self.net.dt, self.net.cs, W0)
        self.tab0 = tables
        self.n0 = n0

    def tau(self, i, n):
        O = self.O
        fi = O.interaction_rows(self.net, self.V, int(n), [int(i)], pair_hi=self.last)[0]
        fs = O.self_rows(self.net, 0, self.delta[: n + 1, : self.n0], int(n), self.tab0, [int(i)])[0]
        return -(self.w.mu / (2 * self.w.cs)) * self.V[n, i] + fs + fi

    def interaction(self, rows, n):
        return self.O.interaction_rows(self.net, self.V, int(n), rows, pair_hi=self.last)

    def self_part(self, rows0, n):
        """The spectral self part at receivers ``rows0`` of fault 0 at step n."""
        return self.O.self_rows(self.net, 0, self.delta[: n + 1, : self.n0], int(n), self.tab0, rows0)

    def interaction_cluster(self, rows, n):
        """The same rows with the cluster-level end truncation (windows per block of the H-matrix partition)."""
        hp = self.w.hparams
        W = self.O.cluster_windows(self.net, int(hp["leaf"]), float(hp["eta_h"]), int(hp.get("max_block", 0)) or 64,
                                   hp["eta_tmax"], hp["max_steps"], no_trunc=bool(hp.get("flags", 0) & 2))
        return self.O.interaction_rows(self.net, self.V, int(n), rows, pair_hi=W)


_WORKER = None


def _worker_init(name, tables):
    global _WORKER
    _WORKER = OracleStepper(synth.WORKLOADS[name](), tables)


def _worker_tau(pair):
    return _WORKER.tau(pair[0], pair[1])


def config_of(w, start, K):
    hp = w.hparams
    return {"workload": w.name, "faults": w.n_faults, "elements": w.N, "steps": w.steps,
            "timed_window": [start, start + K], "batch": 1,
            "leaf": hp["leaf"], "eta_h": hp["eta_h"], "aca_tol": hp["aca_tol"], "eta_tmax": hp["eta_tmax"],
            "eta_w": hp["eta_w"], "q_w": "n_max" if hp["q_w"] <= 0 else hp["q_w"],
            "parallelism": "replicas (independent scenarios per GPU)",
            "l2": "operator larger than L2 (no flush between steps)"}


def run_reference(args, w, start, K, W):
    """The oracle arm: each step evaluates one (element, step) sample of the timed window on the host; the samples
    are spread over the host cores by a spawn process pool (tables built once, shipped to the workers)."""
    import multiprocessing as mp
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    cores = max(1, (os.cpu_count() or 1))
    t0 = time.perf_counter()
    st = OracleStepper(w)
    setup = time.perf_counter() - t0
    elems, steps = oracle_sample(w, start, K, K + W)
    pairs = list(zip(elems.tolist(), steps.tolist()))
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores, initializer=_worker_init, initargs=(w.name, st.tab0)) as pool:
        pool.map(_worker_tau, pairs[:max(W, cores)], chunksize=1)          # warm-up: every worker initialised
        t0 = time.perf_counter()
        pool.map(_worker_tau, pairs[W:], chunksize=4)
        T = time.perf_counter() - t0
    value = K / T
    sample = (f"{K} oracle element-steps (one receiver of fault 0 at a step drawn from the timed window "
              f"[{start}, {start + K}) of the {w.steps}-step run, all lags of every source within the windows, "
              f"NumPy FP64) over a {cores}-process spawn pool; spectral tables of fault 0 built once untimed "
              f"({setup:.1f} s)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
            "steps": K, "warmup": W, "ms_per_step": 1e3 * T / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(w, start, K),
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    return line


# ---------------------------------------------------------------------------------------------------- GPU arm ------

class Clocks:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup(args):
    """One process per GPU (torchrun's RANK / WORLD_SIZE / LOCAL_RANK / MASTER_*); NCCL on GPUs, gloo otherwise.
    The process group only carries the barrier and the max-over-ranks time: scenarios share no data."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        import torch
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        return dist, int(os.environ["RANK"]), world, int(os.environ.get("LOCAL_RANK", "0"))
    return None, 0, 1, 0


def rank_seed(rank: int) -> int:
    """Seed of the scenario a rank runs: independent histories per rank (weak scaling)."""
    return synth.SEED + rank


def job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / seconds


def barrier(dist):
    if dist is not None:
        dist.barrier()


def max_over_ranks(dist, x, device):
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def advance(seas, torch, scn, Vd, n0, n1, device, sample_every=0):
    """Untimed steps n0 .. n1 - 1 (device-resident inputs).  With sample_every > 0, every sample_every-th step is
    also bracketed by CUDA events (its own synchronize), and {step: ms} is returned: the step time as the history
    deepens."""
    t = torch.zeros(Vd.shape[1], dtype=torch.float64, device=device)
    stream = torch.cuda.current_stream(device)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    by_depth = {}
    for n in range(n0, n1):
        sample = sample_every > 0 and n > 0 and n % sample_every == 0
        if sample:
            torch.cuda.synchronize(device)
            a.record(stream)
        seas.seas_push_slip_rate(scn, Vd[n])
        seas.seas_stress_step(scn, t)
        if sample:
            b.record(stream)
            b.synchronize()
            by_depth[n] = a.elapsed_time(b)
    torch.cuda.synchronize(device)
    return by_depth


def nvtx_push(name):
    import torch
    torch.cuda.nvtx.range_push(name)


def nvtx_pop():
    import torch
    torch.cuda.nvtx.range_pop()


def timed_run(seas, torch, scn, Vd, start, K, dist, device):
    """Steps start .. start + K - 1 with device-resident inputs; per-step CUDA events on the library's stream
    (created before the timed region); the parts of the last step are kept."""
    BN = Vd.shape[1]
    tau = torch.zeros((K, BN), dtype=torch.float64, device=device)
    parts = torch.zeros(3 * BN, dtype=torch.float64, device=device)
    stream = torch.cuda.current_stream(device)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    begin, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(dist)
    torch.cuda.synchronize(device)
    nvtx_push("timed")                    # profiler captures select the timed steps by this range
    begin.record(stream)
    for k in range(K):
        ev[k][0].record(stream)
        seas.seas_push_slip_rate(scn, Vd[start + k])
        seas.seas_stress_step(scn, tau[k], parts=parts if k == K - 1 else None)
        ev[k][1].record(stream)
    end.record(stream)
    torch.cuda.synchronize(device)
    nvtx_pop()
    barrier(dist)
    total_ms = begin.elapsed_time(end)
    per = np.array([a.elapsed_time(b) for a, b in ev])
    return total_ms, per, tau, parts.reshape(3, BN)


def roofline_of(timing, batch, peak, fp64_peak, prec):
    """Roofline of the interaction kernel from the library's per-kernel events over a timed window."""
    ms = timing["ms"]
    n_launch = max(1, timing["launches"]["interaction"])
    inter_ms = ms["interaction"] + ms["interaction_source"]          # the two passes of one interaction step
    secs = inter_ms / 1e3
    gbs = timing["interaction_bytes"] / secs / 1e9 if inter_ms > 0 else 0.0
    common = {"kernel": "k_interaction (source pass + receiver pass of one step)",
              "algorithmic_bytes_per_launch": timing["interaction_bytes"] / n_launch,
              "mean_launch_ms": inter_ms / n_launch, "dominant_by_time": max(ms, key=ms.get),
              "pass_ms": {"source": ms["interaction_source"] / n_launch, "receiver": ms["interaction"] / n_launch},
              "kernel_ms": ms, "launches": timing["launches"]}
    if prec == 0:
        # FP64: one FMA per 8 algorithmic bytes per scenario; the FP64 pipe is below the HBM rate
        tflops = 2.0 * timing["interaction_bytes"] / 8 * batch / secs / 1e12 if inter_ms > 0 else 0.0
        roof = {"bound": "alu", "achieved": tflops, "peak": fp64_peak[0], "unit": "TFLOP/s",
                "frac": tflops / fp64_peak[0], "peak_kind": fp64_peak[1],
                "hbm_achieved_gbs": gbs, "hbm_frac": gbs / peak[0]}
    else:
        roof = {"bound": "hbm", "achieved": gbs, "peak": peak[0], "unit": "GB/s", "frac": gbs / peak[0],
                "peak_kind": peak[1]}
    roof.update(common)
    return roof


def rel(a, b):
    nb = float(np.linalg.norm(b))
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.linalg.norm(a))


def run_ours(args, w, start, K, W):
    import torch
    from paper_2603_00383_gb300 import seas
    dist, rank, world, local = dist_setup(args)
    w.seed = rank_seed(rank)                                # independent scenario per rank
    # CPU oracle first (before any GPU work in this process): the CPU baseline and the interaction rows that every
    # storage precision is checked against
    oracle, ref_int, ref_int_cluster, ref_self = None, None, None, None
    rows = oracle_rows(w)
    rows0 = np.linspace(0, int(w.faults[0, 4]) - 1, 8).astype(int)          # receivers of fault 0 (self part)
    if rank == 0 and (args.cpu_sample > 0 or not args.no_oracle_rows):
        t0 = time.perf_counter()
        st = OracleStepper(w)
        log(f"oracle tables {time.perf_counter() - t0:.1f} s")
        if args.cpu_sample > 0:
            elems, steps = oracle_sample(w, start, K, args.cpu_sample)
            t0 = time.perf_counter()
            ref = np.array([st.tau(i, n) for i, n in zip(elems, steps)])
            T = time.perf_counter() - t0
            oracle = (elems, steps, ref, T)
            log(f"cpu baseline {args.cpu_sample} element-steps in {T:.1f} s")
        if not args.no_oracle_rows:
            t0 = time.perf_counter()
            ref_int = st.interaction(rows, w.steps - 1)
            ref_self = st.self_part(rows0, w.steps - 1)
            log(f"oracle interaction and self rows {time.perf_counter() - t0:.1f} s")
            if not args.no_cluster:
                t0 = time.perf_counter()
                ref_int_cluster = st.interaction_cluster(rows, w.steps - 1)
                log(f"oracle interaction rows, cluster-level windows {time.perf_counter() - t0:.1f} s")
        del st
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    stream = torch.cuda.current_stream(device)
    V = w.slip_rate(0, 0, w.steps)
    Vd = torch.from_numpy(V).to(device)
    peak = load_peaks()
    fma = seas.seas_measure_fp64_peak(local)
    fp64_peak = (2.0 * fma / 1e12, "measured: FP64 FMA probe of the library (seas_measure_fp64_peak), "
                                   f"{fma / 1e9:.1f} G FMA/s")
    log(f"fp64 probe {fp64_peak[0]:.3f} TFLOP/s")

    def tau_err(tau_win, elems_steps=None):
        if oracle is None:
            return None
        elems, steps, ref, _ = oracle
        got = tau_win.cpu().numpy()[steps - start, elems]
        return rel(got, ref)

    def int_err(parts_last, b=0, ref=None):
        r = ref_int if ref is None else ref
        if r is None:
            return None
        return rel(parts_last[2, b * w.N + rows].cpu().numpy(), r)

    # consumer warps per interaction pass picked by the library's autotuner for every measured scenario; copies of a
    # scenario (same operator and batch) take the choice from this run's cache file
    tune_cache = os.path.join(tempfile.mkdtemp(prefix="seas_tune_"), "choices.txt")

    def session(prec, batch=1, flags=None):
        extra = {} if flags is None else {"flags": flags}
        t0 = time.perf_counter()
        s = seas.Session(w, batch=batch, device=local, stream=stream.cuda_stream, precision=prec, **extra)
        log(f"build prec {prec} batch {batch} flags {flags}: {time.perf_counter() - t0:.1f} s, "
            f"{s.stats['bytes_interaction'] / 1e9:.2f} GB")
        s.tune = seas.seas_scenario_autotune(s.scn, tune_cache, reps=5)
        log(f"autotune: consumer warps {s.tune['consumer_warps']} (median ms {s.tune['ms']})")
        return s

    def measure(s, Vx, batch, prec, clocks=False):
        """Advance to the window and time it as the step runs (no per-kernel events: the self-term convolution
        overlaps the interaction); then repeat the window on a checkpoint copy with per-kernel events for the
        roofline."""
        t0 = time.perf_counter()
        advance(seas, torch, s.scn, Vx, 0, start, device)
        log(f"advance {start} steps: {time.perf_counter() - t0:.1f} s")
        cdir = tempfile.mkdtemp(prefix="seas_leg_")
        cpath = os.path.join(cdir, "window_start.ckpt")
        seas.seas_scenario_save(s.scn, cpath)
        if clocks:
            with Clocks(local) as clk:
                total_ms, per, tau, parts = timed_run(seas, torch, s.scn, Vx, start, K, dist, device)
            clk_summary = clk.summary()
        else:
            total_ms, per, tau, parts = timed_run(seas, torch, s.scn, Vx, start, K, dist, device)
            clk_summary = None
        seas.seas_scenario_check(s.scn)                  # raises if a bounded device wait ran out
        copy = seas.seas_scenario_load(s.op, cpath)
        os.remove(cpath)
        os.rmdir(cdir)
        seas.seas_scenario_autotune(copy, tune_cache, reps=1)
        seas.seas_scenario_set_timing(copy, True)
        timed_run(seas, torch, copy, Vx, start, K, dist, device)
        seas.seas_scenario_check(copy)
        timing = seas.seas_scenario_get_timing(copy)
        seas.seas_destroy_scn(copy)
        total_ms = max_over_ranks(dist, total_ms, device)
        return {"total_ms": total_ms, "per": per, "tau": tau, "parts": parts, "timing": timing,
                "roofline": roofline_of(timing, batch, peak, fp64_peak, prec), "clocks": clk_summary}

    if args.batched_only:
        return run_batched_only(args, w, start, K, seas, torch, session, measure, device, rows, int_err, world)
    # ---- headline: scenario A (no kernel timing) for value and latency; B, a copy of A's state at the window's
    # start, for the per-kernel events of the roofline; C, another copy, end to end through host buffers
    head_code, head_dtype = PRECISIONS[args.precision]
    s = session(head_code)
    t0 = time.perf_counter()
    by_depth = advance(seas, torch, s.scn, Vd, 0, start, device, sample_every=max(1, w.steps // 10))
    log(f"advance {start} steps: {time.perf_counter() - t0:.1f} s; ms per step by depth {by_depth}")
    ckpt_dir = tempfile.mkdtemp(prefix="seas_bench_")
    ckpt = os.path.join(ckpt_dir, "window_start.ckpt")
    seas.seas_scenario_save(s.scn, ckpt)
    with Clocks(local) as clk:
        total_ms, per, tau, parts = timed_run(seas, torch, s.scn, Vd, start, K, dist, device)
    clocks = clk.summary()
    seas.seas_scenario_check(s.scn)
    total_ms = max_over_ranks(dist, total_ms, device)
    value = job_rate(w.N * K, world, total_ms / 1e3)
    err_tau = tau_err(tau)
    err_int = int_err(parts)
    err_self = None if ref_self is None else rel(parts[1, rows0].cpu().numpy(), ref_self)
    err_rad = rel(parts[0].cpu().numpy(), -(w.mu / (2 * w.cs)) * V[w.steps - 1])
    log(f"headline {value / 1e6:.3f} M element-steps/s, p50 {np.percentile(per, 50):.3f} ms")

    sB = seas.seas_scenario_load(s.op, ckpt)
    seas.seas_scenario_autotune(sB, tune_cache, reps=1)       # the headline's choice, from the cache
    seas.seas_scenario_set_timing(sB, True)
    _, perB, tauB, _ = timed_run(seas, torch, sB, Vd, start, K, dist, device)
    seas.seas_scenario_check(sB)
    timing = seas.seas_scenario_get_timing(sB)
    seas.seas_destroy_scn(sB)
    roofline = roofline_of(timing, 1, peak, fp64_peak, head_code)
    roofline["timed_with"] = ("per-kernel CUDA events on the library's stream over the same step window, in a "
                              "copy of the scenario taken at the window's start (the headline run records none)")
    if not torch.equal(tauB, tau):
        log("warning: kernel-timing pass differs from the headline run")
    # the same window replayed as a captured CUDA graph: one graph launch per step (the step's seven kernels, the
    # self-term convolution on its forked branch), the slip rate copied into the graph's input buffer each step
    sG = seas.seas_scenario_load(s.op, ckpt)
    seas.seas_scenario_autotune(sG, tune_cache, reps=1)
    vG = torch.zeros(w.N, dtype=torch.float64, device=device)
    tG = torch.zeros(w.N, dtype=torch.float64, device=device)
    seas.seas_scenario_graph_create(sG, vG, tG)
    evG = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    torch.cuda.synchronize(device)
    for k in range(K):
        evG[k][0].record(stream)
        vG.copy_(Vd[start + k])
        seas.seas_scenario_graph_step(sG)
        evG[k][1].record(stream)
    torch.cuda.synchronize(device)
    seas.seas_scenario_check(sG)
    perG = np.array([a_.elapsed_time(b_) for a_, b_ in evG])
    graph = {"ms_per_step": float(perG.mean()), "p50_ms": float(np.percentile(perG, 50)),
             "value": job_rate(w.N * K, world, float(perG.sum()) / 1e3), "unit": METRIC,
             "last_step_equal": bool(torch.equal(tG, tau[K - 1]))}
    seas.seas_destroy_scn(sG)
    log(f"graph replay: {graph['ms_per_step']:.3f} ms per step (eager {total_ms / K:.3f})")
    if args.dump_step_bytes and rank == 0:
        with open(args.dump_step_bytes, "w") as fh:
            json.dump({"precision": args.precision, "steps": w.steps,
                       "bytes": [seas.seas_op_step_bytes(s.op, n) for n in range(w.steps)]}, fh)
    window_bytes = float(np.mean([seas.seas_op_step_bytes(s.op, n) for n in range(start, start + K)]))

    e2e = None
    if not args.no_e2e:
        sC = seas.seas_scenario_load(s.op, ckpt)
        seas.seas_scenario_autotune(sC, tune_cache, reps=1)
        Vh = torch.from_numpy(V).pin_memory().numpy()
        th = torch.zeros(w.N, dtype=torch.float64).pin_memory().numpy()
        barrier(dist)
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        for k in range(K):
            seas.seas_push_slip_rate(sC, Vh[start + k])
            seas.seas_stress_step(sC, th)
        torch.cuda.synchronize(device)
        barrier(dist)
        e2e_s = max_over_ranks(dist, time.perf_counter() - t0, device)
        seas.seas_destroy_scn(sC)
        e2e = {"value": w.N * K * world / e2e_s, "unit": METRIC, "h2d_bytes_per_step": w.N * 8,
               "d2h_bytes_per_step": w.N * 8, "last_step_equal": bool(np.array_equal(th, tau[-1].cpu().numpy()))}
    os.unlink(ckpt)
    os.rmdir(ckpt_dir)

    variants = {}
    if not args.no_variants:
        for name, (code, dtype) in PRECISIONS.items():
            if name == args.precision:
                continue
            s2 = session(code)
            r2 = measure(s2, Vd, 1, code)
            variants[name] = {"value": job_rate(w.N * K, world, r2["total_ms"] / 1e3), "unit": METRIC,
                              "dtype": dtype, "ms_per_step": r2["total_ms"] / K,
                              "p50_ms": float(np.percentile(r2["per"], 50)),
                              "p99_ms": float(np.percentile(r2["per"], 99)),
                              "rel_l2_interaction_vs_oracle": int_err(r2["parts"]),
                              "rel_l2_tau_vs_oracle": tau_err(r2["tau"]),
                              "rel_l2_interaction_vs_headline": rel(r2["parts"][2].cpu().numpy(),
                                                                    parts[2].cpu().numpy()),
                              "rel_l2_tau_vs_headline": rel(r2["tau"].cpu().numpy(), tau.cpu().numpy()),
                              "bytes_interaction": s2.stats["bytes_interaction"],
                              "consumer_warps": s2.tune["consumer_warps"],
                              "roofline": {k: r2["roofline"][k] for k in (
                                  "bound", "achieved", "peak", "unit", "frac", "mean_launch_ms", "pass_ms")}}
            s2.close()
            del r2

    # batched ensemble: 8 scenarios (independent seeded histories, scenario 0 = the headline's) share one operator;
    # one persistent interaction kernel per step serves all 8 with each operator byte read once
    batched = {}
    if not args.no_batched:
        B = 8
        V8 = np.stack([w.slip_rate(b, 0, w.steps) for b in range(B)], axis=1).reshape(w.steps, B * w.N)
        V8d = torch.from_numpy(V8).to(device)
        del V8
        for name in ("bf16", "fp64"):
            code, dtype = PRECISIONS[name]
            s3 = session(code, batch=B)
            r3 = measure(s3, V8d, B, code)
            t0 = r3["tau"][:, : w.N]
            batched[name] = {"value": job_rate(B * w.N * K, world, r3["total_ms"] / 1e3), "unit": METRIC,
                             "batch": B, "dtype": dtype, "ms_per_step": r3["total_ms"] / K,
                             "p50_ms": float(np.percentile(r3["per"], 50)),
                             "p99_ms": float(np.percentile(r3["per"], 99)),
                             "rel_l2_member0_interaction_vs_oracle": int_err(r3["parts"], 0),
                             "rel_l2_member0_tau_vs_headline": rel(t0.cpu().numpy(), tau.cpu().numpy()),
                             "consumer_warps": s3.tune["consumer_warps"],
                             "roofline": {k: r3["roofline"][k] for k in (
                                 "bound", "achieved", "peak", "unit", "frac", "mean_launch_ms", "pass_ms")}}
            s3.close()
            del r3
        del V8d

    # the flagged static tail (elastostatic response of the history the windows drop) on the headline operator
    tail, tail_tau = None, None
    if not args.no_tail:
        s4 = session(head_code, flags=int(w.hparams.get("flags", 0)) | seas.SEAS_FLAG_STATIC_TAIL)
        r4 = measure(s4, Vd, 1, head_code)
        tv = job_rate(w.N * K, world, r4["total_ms"] / 1e3)
        tail = {"value": tv, "unit": METRIC, "ms_per_step": r4["total_ms"] / K, "cost_vs_headline": value / tv - 1,
                "tail_share_of_tau": rel(r4["tau"].cpu().numpy(), tau.cpu().numpy())}
        tail_tau = r4["tau"].cpu().numpy()
        s4.close()
        del r4

    # cluster-level end truncation (Sec. 4.3): the headline operator with a window per H-matrix block
    cluster = None
    if not args.no_cluster:
        s5 = session(head_code, flags=int(w.hparams.get("flags", 0)) | seas.SEAS_FLAG_CLUSTER_TRUNC)
        r5 = measure(s5, Vd, 1, head_code)
        cv = job_rate(w.N * K, world, r5["total_ms"] / 1e3)
        cluster = {"value": cv, "unit": METRIC, "ms_per_step": r5["total_ms"] / K,
                   "p50_ms": float(np.percentile(r5["per"], 50)), "speedup": cv / value,
                   "bytes_interaction": s5.stats["bytes_interaction"],
                   "bytes_vs_headline": s5.stats["bytes_interaction"] / s.stats["bytes_interaction"],
                   "window_bytes_per_step": r5["roofline"]["algorithmic_bytes_per_launch"],
                   "rel_l2_interaction_vs_oracle": int_err(r5["parts"], ref=ref_int_cluster),
                   "rel_l2_interaction_vs_headline": rel(r5["parts"][2].cpu().numpy(), parts[2].cpu().numpy()),
                   "rel_l2_tau_vs_headline": rel(r5["tau"].cpu().numpy(), tau.cpu().numpy()),
                   "consumer_warps": s5.tune["consumer_warps"],
                   "roofline": {k: r5["roofline"][k] for k in (
                       "bound", "achieved", "peak", "unit", "frac", "mean_launch_ms", "pass_ms")}}
        log(f"cluster-level truncation {cv / 1e6:.3f} M element-steps/s ({cv / value:.2f}x), "
            f"{cluster['bytes_vs_headline']:.3f} of the operator bytes")
        s5.close()
        del r5
        if tail_tau is not None:
            # with the static tail per block: against the fault-pair windows with their tail
            s6 = session(head_code, flags=int(w.hparams.get("flags", 0)) | seas.SEAS_FLAG_CLUSTER_TRUNC
                         | seas.SEAS_FLAG_STATIC_TAIL)
            r6 = measure(s6, Vd, 1, head_code)
            cluster["with_static_tail"] = {
                "value": job_rate(w.N * K, world, r6["total_ms"] / 1e3), "unit": METRIC,
                "ms_per_step": r6["total_ms"] / K,
                "rel_l2_tau_vs_pair_windows_with_tail": rel(r6["tau"].cpu().numpy(), tail_tau)}
            s6.close()
            del r6

    # a fault breaking a traction-free surface (method of images), the shape of App. B's single-fault check: the
    # self term of the doubled 3200-element fault per step (no interaction), the deepest K steps of 2000
    surface = None
    if not args.no_surface:
        ws = synth.surface_fault_1600(steps=w.steps)
        Vs = torch.from_numpy(ws.slip_rate(0, 0, ws.steps)).to(device)
        ss = seas.Session(ws, device=local, stream=stream.cuda_stream)
        s0 = ws.steps - K
        advance(seas, torch, ss.scn, Vs, 0, s0, device)
        ms_s, per_s, _, _ = timed_run(seas, torch, ss.scn, Vs, s0, K, dist, device)
        seas.seas_scenario_check(ss.scn)
        ms_s = max_over_ranks(dist, ms_s, device)
        surface = {"workload": ws.name, "elements": ws.N, "elements_with_images": 2 * ws.N, "steps": ws.steps,
                   "timed_window": [s0, s0 + K], "value": job_rate(ws.N * K, world, ms_s / 1e3), "unit": METRIC,
                   "ms_per_step": ms_s / K, "p50_ms": float(np.percentile(per_s, 50)),
                   "bytes_self": ss.stats["bytes_self"],
                   "parity": "against the oracle's doubled network at 64 and 2 x 40 elements (GPU tests)"}
        log(f"surface fault {surface['value'] / 1e6:.3f} M element-steps/s, {ms_s / K:.3f} ms per step")
        ss.close()
        del Vs

    # plain FP64 GPU path: every block dense (leaf blocks, exact windows), no compression, FP64 arithmetic
    plain = None
    if not args.no_plain:
        p = session(0, flags=seas.SEAS_FLAG_DENSE)
        rp = measure(p, Vd, 1, 0)
        pv = job_rate(w.N * K, world, rp["total_ms"] / 1e3)
        plain = {"value": pv, "unit": METRIC, "ms_per_step": rp["total_ms"] / K,
                 "p50_ms": float(np.percentile(rp["per"], 50)), "p99_ms": float(np.percentile(rp["per"], 99)),
                 "speedup": value / pv, "bytes_interaction": p.stats["bytes_interaction"],
                 "rel_l2_interaction_vs_oracle": int_err(rp["parts"]), "rel_l2_tau_vs_oracle": tau_err(rp["tau"]),
                 "rel_l2_tau_vs_headline": rel(tau.cpu().numpy(), rp["tau"].cpu().numpy())}
        p.close()
        del rp

    served = run_served(args, dist, local) if args.served_seconds > 0 and rank == 0 else None
    ensemble = run_ensemble88(args, dist, local, K, peak, world) if not args.no_ensemble else None

    roofline["traffic"] = None
    tf = os.path.join(ROOT, "profiles", "interaction_traffic.json")
    if os.path.exists(tf):
        with open(tf) as fh:
            tr = json.load(fh)
        ratio = tr.get("dram_over_algorithmic", {}).get(args.precision)
        if tr.get("kernel_version") == seas_kernel_version() and ratio is not None:
            # DRAM bytes of the captured launch over its algorithmic bytes, scaled to this window's mean launch
            roofline["traffic"] = ratio * roofline["algorithmic_bytes_per_launch"]

    line = None
    if rank == 0:
        cpu = None
        if oracle is not None:
            cpu = {"value": args.cpu_sample / oracle[3], "unit": METRIC, "cores": 1, "kind": "oracle",
                   "sample": f"{args.cpu_sample} element-steps (receivers of fault 0 at steps spread over the timed "
                             f"window [{start}, {start + K}), all lags of all sources within the windows, NumPy "
                             f"FP64, one thread), {oracle[3]:.1f} s"}
        launches = timing["launches"]
        stats = s.stats
        line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": K, "warmup": W,
                "ms_per_step": total_ms / K, "p50_ms": float(np.percentile(per, 50)),
                "p99_ms": float(np.percentile(per, 99)),
                "ms_by_history_depth": {str(k): v for k, v in by_depth.items()},
                "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": head_dtype, "data": "synthetic",
                "config": dict(config_of(w, start, K), precision=args.precision,
                               window_algorithmic_bytes_per_step=window_bytes),
                "rel_l2_tau_vs_oracle": err_tau, "rel_l2_interaction_vs_oracle": err_int,
                "rel_l2_self_vs_oracle": err_self, "rel_l2_radiation_vs_oracle": err_rad,
                "oracle_rows": {"interaction": [int(r) for r in rows], "self": [int(r) for r in rows0],
                                "step": w.steps - 1},
                "operator": {k: stats[k] for k in (
                    "n_blocks_far", "n_blocks_near", "compression_ratio", "bytes_interaction", "mean_rank",
                    "max_rank", "build_seconds", "n_tasks")},
                "vs_plain_fp64_gpu": plain, "variants": variants, "batched": batched, "static_tail": tail,
                "cluster_trunc": cluster, "surface_fault": surface, "e2e": e2e,
                "served": served, "ensemble_8x8": ensemble, "graph": graph,
                "roofline": roofline, "cpu_baseline": cpu, "clocks": clocks,
                "autotune": {"consumer_warps": s.tune["consumer_warps"], "median_launch_ms": s.tune["ms"],
                             "by": "seas_scenario_autotune (per pass, every task active, 5 launches each)"},
                "gpu_launches": int(sum(launches.values()))}
    s.close()
    if dist is not None:
        dist.destroy_process_group()
    return line


def run_batched_only(args, w, start, K, seas, torch, session, measure, device, rows, int_err, world):
    """The 8-scenario ensemble legs alone (profiling captures of the batched kernels)."""
    B = 8
    V8 = np.stack([w.slip_rate(b, 0, w.steps) for b in range(B)], axis=1).reshape(w.steps, B * w.N)
    V8d = torch.from_numpy(V8).to(device)
    out = {}
    for name in ("bf16", "fp64"):
        code, dtype = PRECISIONS[name]
        s3 = session(code, batch=B)
        r3 = measure(s3, V8d, B, code)
        out[name] = {"value": job_rate(B * w.N * K, world, r3["total_ms"] / 1e3), "ms_per_step": r3["total_ms"] / K,
                     "roofline": {k: r3["roofline"][k] for k in ("bound", "achieved", "frac", "mean_launch_ms",
                                                                   "pass_ms")}}
        s3.close()
    return {"batched_only": out, "config": config_of(w, start, K)}


def run_ensemble88(args, dist, local, K, peak, world):
    """Batched ensemble: 64 scenarios over 8 seeded geometries (2..12 faults, 500..6000 elements, 1000..5000 steps),
    8 scenarios with independent slip-rate histories per geometry sharing its BF16 operator in one scenario batch
    (tensor-core consumers).  Each geometry is advanced untimed to its K deepest steps, which are timed; the value
    is the element-steps of all 64 scenarios over the summed timed time of the 8 batches (run one after another)."""
    import torch
    from paper_2603_00383_gb300 import seas
    code, dtype = PRECISIONS["bf16"]
    device = torch.device("cuda", local)
    stream = torch.cuda.current_stream(device)
    total_ms, units, inter_ms, inter_bytes, per = 0.0, 0, 0.0, 0, []
    t_all = time.perf_counter()
    tune_cache = os.path.join(tempfile.mkdtemp(prefix="seas_tune_"), "choices.txt")
    for g in range(8):
        w = synth.ensemble_network(g)
        start, k = window(w, K)
        B = 8
        s = seas.Session(w, batch=B, device=local, stream=stream.cuda_stream, precision=code)
        seas.seas_scenario_autotune(s.scn, tune_cache, reps=3)
        Vd = torch.from_numpy(np.stack([w.slip_rate(b, 0, w.steps) for b in range(B)], axis=1).reshape(
            w.steps, B * w.N)).to(device)
        advance(seas, torch, s.scn, Vd, 0, start, device)
        # the window as the step runs (no per-kernel events), then again on a checkpoint copy with events
        cdir = tempfile.mkdtemp(prefix="seas_ens_")
        cpath = os.path.join(cdir, "window_start.ckpt")
        seas.seas_scenario_save(s.scn, cpath)
        ms, pstep, _, _ = timed_run(seas, torch, s.scn, Vd, start, k, dist, device)
        seas.seas_scenario_check(s.scn)
        copy = seas.seas_scenario_load(s.op, cpath)
        os.remove(cpath)
        os.rmdir(cdir)
        seas.seas_scenario_autotune(copy, tune_cache, reps=1)
        seas.seas_scenario_set_timing(copy, True)
        timed_run(seas, torch, copy, Vd, start, k, dist, device)
        seas.seas_scenario_check(copy)
        tm = seas.seas_scenario_get_timing(copy)
        seas.seas_destroy_scn(copy)
        total_ms += ms
        units += B * w.N * k
        inter_ms += tm["ms"]["interaction"] + tm["ms"]["interaction_source"]
        inter_bytes += tm["interaction_bytes"]
        per.append({"geometry": g, "faults": w.n_faults, "elements": w.N, "steps": w.steps,
                    "ms_per_step": ms / k, "p50_ms": float(np.percentile(pstep, 50)),
                    "bytes_interaction": s.stats["bytes_interaction"]})
        s.close()
        del Vd
    log(f"ensemble 8x8: {time.perf_counter() - t_all:.1f} s, {units / (total_ms / 1e3) / 1e6:.2f} M element-steps/s")
    gbs = inter_bytes / (inter_ms / 1e3) / 1e9 if inter_ms > 0 else 0.0
    total_ms = max_over_ranks(dist, total_ms, device)
    return {"value": job_rate(units, world, total_ms / 1e3), "unit": METRIC, "dtype": dtype, "scenarios": 64,
            "timed_steps_per_geometry": K, "geometries": per,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak[0], "unit": "GB/s", "frac": gbs / peak[0]}}


SERVED = dict(pool=8, rate=20.0, steps_lo=1000, steps_hi=20000, lag_cap=500, batch=8, budget=24 << 30,
              precision="bf16")


def run_served(args, dist, local):
    """Served workload: Poisson arrivals (20 per second) of scenario requests on a pool of 8 seeded networks of
    256..8000 elements (log-uniform), 1000..20000 steps each (log-uniform), BF16 operators with windows capped at
    500 lags, slot groups of 8 members, an HBM budget of 24 GiB.  The operators are built before the window (warm
    start); the server then runs the arrival trace for --served-seconds of wall time.  Throughput counts the steps
    completed in that window; latency is each request-step's group tick (CUDA events on the group's stream)."""
    import torch
    from paper_2603_00383_gb300 import seas, serve
    cfg = dict(SERVED)
    code, dtype = PRECISIONS[cfg["precision"]]
    geoms = [synth.served_network(g, max_steps=cfg["lag_cap"], precision=code) for g in range(cfg["pool"])]
    trace = serve.poisson_trace(cfg["pool"], cfg["rate"], args.served_seconds, cfg["steps_lo"], cfg["steps_hi"])
    srv = serve.Server(geoms, budget=cfg["budget"], batch=cfg["batch"], device=local, precision=code)
    t0 = time.perf_counter()
    srv.prebuild(range(cfg["pool"]))
    torch.cuda.synchronize(local)
    log(f"served: warm start {time.perf_counter() - t0:.1f} s, "
        f"builds {[round(x, 1) for x in srv.backend.build_seconds.values()]} s")
    with Clocks(local) as clk:
        wall = srv.run(trace, until=args.served_seconds)
    torch.cuda.synchronize(local)
    reqs = list(srv.sched.requests.values())
    lat = np.array(srv.latency_ms) if srv.latency_ms else np.zeros(1)
    waits = [r.admitted - r.arrival for r in reqs if r.admitted is not None]
    out = {"value": srv.element_steps / wall, "unit": METRIC, "dtype": dtype, "wall_s": wall,
           "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
           "request_steps": len(srv.latency_ms), "group_ticks": srv.ticks,
           "requests": {"arrived": len(trace), "admitted": sum(r.admitted is not None for r in reqs),
                        "completed": sum(r.state == "done" for r in reqs),
                        "rejected": sum(r.state == "rejected" for r in reqs)},
           "queue_wait_p50_s": float(np.percentile(waits, 50)) if waits else None,
           "queue_wait_p99_s": float(np.percentile(waits, 99)) if waits else None,
           "pool_elements": [w.N for w in geoms], "hbm_held_gb": srv.sched.used / 1e9,
           "config": {k: v for k, v in cfg.items() if k != "budget"} | {"budget_gib": cfg["budget"] >> 30},
           "clocks": clk.summary()}
    log(f"served: {out['value'] / 1e6:.2f} M element-steps/s, p50 {out['p50_ms']:.3f} ms, p99 {out['p99_ms']:.3f} ms,"
        f" {out['requests']}")
    for g in list(srv.backend.op):
        for gid in [gid for gid, G in srv.backend.groups.items() if G["geom"] == g]:
            srv.backend.drop(gid)
        srv.backend.evict(g)
    return out


def seas_kernel_version():
    """Hash of the interaction kernel's source (seas_step.cu from its section header up to the next kernel), so
    that profiled DRAM counters are used only for the kernel they were taken on."""
    import hashlib
    with open(os.path.join(ROOT, "paper_2603_00383_gb300", "csrc", "seas_step.cu")) as fh:
        text = fh.read()
    a = text.index("// Space-time interaction")
    b = min(i for i in (text.find("// Static tail of the interaction"),
                        text.index("// f_int[b][e] = sum over the blocks")) if i > a)
    region = text[a:b]
    # the tensor-core consumers are compiled only into the BF16 8-scenario instantiation: not part of the others
    while "// [tensor-core consumers: begin]" in region:
        i = region.rindex("\n", 0, region.index("// [tensor-core consumers: begin]")) + 1
        j = region.index("\n", region.index("// [tensor-core consumers: end]", i)) + 1
        region = region[:i] + region[j:]
    return hashlib.sha1(region.encode()).hexdigest()[:12]


def main():
    args = parse()
    w = synth.WORKLOADS[args.workload]() if args.max_steps is None else synth.WORKLOADS[args.workload](
        steps=args.max_steps)
    start, K = window(w, args.steps)
    W = max(3, args.warmup)
    if args.impl == "reference":
        line = run_reference(args, w, start, K, W)
    else:
        from paper_2603_00383_gb300 import build
        build.build()
        line = run_ours(args, w, start, K, W)
    if line is not None:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
