"""Benchmark of the per-step stress-transfer functional on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload six_fault_3072]

A step is one push of the slip rate plus one seas_stress_step (all hot-path stages: push, forward FFT, mode
convolution, H-matrix interaction, inverse FFT + assembly) on the six-fault, 3072-element network with the
selective H-matrix (leaf 32, eta_H 2, ACA 1e-6) and causal / spectral windows; the timed K steps are the first K
steps of a fresh scenario (K = 2000 is the whole workload).  Prints one JSON line.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

if "--impl" in sys.argv and "reference" in sys.argv:      # the oracle arm runs single-threaded on the host
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ.setdefault(var, "1")

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2603_00383_gb300 import synth  # noqa: E402

METRIC = "element-steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None)
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
    ap.add_argument("--dump-step-bytes", default=None, help="write the per-step algorithmic interaction bytes here")
    return ap.parse_args()


# name -> (seas precision code, dtype label of the arithmetic)
# FP64 pipe of GB300: 152 SMs x 2 FP64 FMA per clock x 2 flops at the 2070 MHz maximum SM clock
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2070e6 / 1e12
FP64_PEAK_KIND = "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2070 MHz"
PRECISIONS = {"fp64": (0, "f64"), "df64": (3, "df64 (fp32 pairs)"), "bf16": (1, "bf16 storage, f32 compensated"),
              "fp16s": (2, "fp16 storage with per-slice scale, f32 compensated")}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------------------------------------ oracle sample --

def oracle_sample(w, K, count, seed=11):
    """(element, step) pairs of the CPU-baseline / reference sample: elements of fault 0 (whose spectral tables the
    oracle builds once, untimed), steps spread over the run so the mean history depth is that of the workload."""
    n0 = int(w.faults[0, 4])
    k = np.arange(count)
    elems = (k * 97 + seed) % n0
    steps = (k * 7919 + 13 * seed) % K
    return elems, steps


class OracleStepper:
    """Evaluates tau at single (element, step) pairs with the CPU oracle (interaction row + spectral self term of
    fault 0 + radiation damping), with the workload's windows."""

    def __init__(self, w, K, tables=None):
        from oracle import seas_oracle as O
        self.O = O
        self.w = w
        self.net = O.network(w.faults, w.mu, w.cs)
        hp = w.hparams
        self.V = w.slip_rate(0, 0, K)
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


_WORKER = None


def _worker_init(name, K, tables):
    global _WORKER
    _WORKER = OracleStepper(synth.WORKLOADS[name](), K, tables)


def _worker_tau(pair):
    return _WORKER.tau(pair[0], pair[1])


def run_reference(args, w, K, W):
    """The oracle arm: each step evaluates one (element, step) sample of the workload on the host; the samples are
    spread over the host cores by a spawn process pool (tables built once, shipped to the workers)."""
    import multiprocessing as mp
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    cores = max(1, (os.cpu_count() or 1))
    t0 = time.perf_counter()
    st = OracleStepper(w, K)
    setup = time.perf_counter() - t0
    elems, steps = oracle_sample(w, K, K + W)
    pairs = list(zip(elems.tolist(), steps.tolist()))
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores, initializer=_worker_init, initargs=(w.name, K, st.tab0)) as pool:
        pool.map(_worker_tau, pairs[:max(W, cores)], chunksize=1)          # warm-up: every worker initialised
        t0 = time.perf_counter()
        pool.map(_worker_tau, pairs[W:], chunksize=4)
        T = time.perf_counter() - t0
    value = K / T
    sample = (f"{K} oracle element-steps (one receiver of fault 0 at a step drawn uniformly from the {K}-step run, "
              f"all lags of every source, NumPy FP64) over a {cores}-process spawn pool; spectral tables of fault 0 "
              f"built once untimed ({setup:.1f} s)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": args.gpus,
            "steps": K, "warmup": W, "ms_per_step": 1e3 * T / K, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(w, K),
            "cpu_baseline": {"value": value, "unit": METRIC, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    return line


def config_of(w, K):
    hp = w.hparams
    return {"workload": w.name, "faults": w.n_faults, "elements": w.N, "steps": K, "batch": 1,
            "leaf": hp["leaf"], "eta_h": hp["eta_h"], "aca_tol": hp["aca_tol"], "eta_tmax": hp["eta_tmax"],
            "eta_w": hp["eta_w"], "q_w": "n_max" if hp["q_w"] <= 0 else hp["q_w"],
            "parallelism": "replicas (independent scenarios per GPU)",
            "l2": "operator larger than L2 (no flush between steps)"}


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


def timed_run(seas, torch, s, Vd, K, dist, device, out_tau=None):
    """K steps with device-resident inputs; per-step CUDA events on the library's stream."""
    N = Vd.shape[1]
    tau = out_tau if out_tau is not None else torch.zeros((K, N), dtype=torch.float64, device=device)
    stream = torch.cuda.current_stream(device)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(dist)
    torch.cuda.synchronize(device)
    start.record(stream)
    for n in range(K):
        ev[n][0].record(stream)
        seas.seas_push_slip_rate(s.scn, Vd[n])
        seas.seas_stress_step(s.scn, tau[n])
        ev[n][1].record(stream)
    stop.record(stream)
    torch.cuda.synchronize(device)
    barrier(dist)
    total_ms = start.elapsed_time(stop)
    per = np.array([a.elapsed_time(b) for a, b in ev])
    return total_ms, per, tau


def run_precision(seas, torch, wr, prec, Vd, K, W, dist, device, stream, peak, batch=1, flags=None):
    """Builds the operator in one storage precision and times K steps of `batch` scenarios sharing it (Vd is
    [K][batch * N]); returns the measurements and tau."""
    extra = {} if flags is None else {"flags": flags}
    s = seas.Session(wr, batch=batch, device=device.index, stream=stream.cuda_stream, precision=prec, **extra)
    warm = seas.seas_scenario_create(s.op, batch)
    tw = torch.zeros(batch * wr.N, dtype=torch.float64, device=device)
    for n in range(W):
        seas.seas_push_slip_rate(warm, Vd[n % K])
        seas.seas_stress_step(warm, tw)
    torch.cuda.synchronize(device)
    seas.seas_destroy_scn(warm)
    seas.seas_scenario_set_timing(s.scn, True)
    with Clocks(device.index) as clk:
        total_ms, per, tau = timed_run(seas, torch, s, Vd, K, dist, device)
    seas.seas_scenario_check(s.scn)                      # raises if a bounded device wait ran out
    timing = seas.seas_scenario_get_timing(s.scn)
    total_ms = max_over_ranks(dist, total_ms, device)
    ms = timing["ms"]
    launches = timing["launches"]
    n_launch = max(1, launches["interaction"])
    inter_ms = ms["interaction"]
    secs = inter_ms / 1e3
    achieved = timing["interaction_bytes"] / secs / 1e9 if inter_ms > 0 else 0.0
    common = {"kernel": "k_interaction", "algorithmic_bytes_per_launch": timing["interaction_bytes"] / n_launch,
              "mean_launch_ms": inter_ms / n_launch, "dominant_by_time": max(ms, key=ms.get), "kernel_ms": ms}
    if prec == 0:
        # FP64: one FMA per 8 algorithmic bytes per scenario; the FP64 pipe (2 FMA/clk/SM) is below the HBM rate
        tflops = 2.0 * timing["interaction_bytes"] / 8 * s.scn.B / secs / 1e12 if inter_ms > 0 else 0.0
        roof = {"bound": "alu", "achieved": tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": tflops / FP64_PEAK_TFLOPS, "peak_kind": FP64_PEAK_KIND,
                "hbm_achieved_gbs": achieved, "hbm_frac": achieved / peak[0]}
    else:
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak[0], "unit": "GB/s", "frac": achieved / peak[0],
                "peak_kind": peak[1]}
    roof.update(common)
    res = {"total_ms": total_ms, "per": per, "stats": s.stats, "timing": timing, "clocks": clk.summary(),
           "roofline": roof}
    s_keep = s
    return res, tau, s_keep


def run_ours(args, w, K, W):
    import torch
    from paper_2603_00383_gb300 import seas
    dist, rank, world, local = dist_setup(args)
    wr = synth.six_fault_3072(steps=K) if w.name == "six_fault_3072" else w
    wr.seed = rank_seed(rank)                            # independent scenario per rank
    # CPU oracle sample first (before any GPU work in this process)
    oracle = None
    if rank == 0 and args.cpu_sample > 0:
        st = OracleStepper(wr, K)
        elems, steps = oracle_sample(wr, K, args.cpu_sample)
        t0 = time.perf_counter()
        ref = np.array([st.tau(i, n) for i, n in zip(elems, steps)])
        T = time.perf_counter() - t0
        oracle = (elems, steps, ref, T)
        del st
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    stream = torch.cuda.current_stream(device)
    V = wr.slip_rate(0, 0, K)
    Vd = torch.from_numpy(V).to(device)
    peak = load_peaks()

    def err_of(tau):
        if oracle is None:
            return None
        elems, steps, ref, _ = oracle
        got = tau.cpu().numpy()[steps, elems]
        return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))

    head_code, head_dtype = PRECISIONS[args.precision]
    res, tau, s = run_precision(seas, torch, wr, head_code, Vd, K, W, dist, device, stream, peak)
    if args.dump_step_bytes and rank == 0:
        # algorithmic interaction bytes of every step, to match profiled launches to steps
        with open(args.dump_step_bytes, "w") as fh:
            json.dump({"precision": args.precision, "steps": K,
                       "bytes": [seas.seas_op_step_bytes(s.op, n) for n in range(K)]}, fh)
    value = job_rate(wr.N * K, world, res["total_ms"] / 1e3)
    err = err_of(tau)
    stats = res["stats"]

    variants = {}
    if not args.no_variants:
        for name, (code, dtype) in PRECISIONS.items():
            if name == args.precision:
                continue
            r2, tau2, s2 = run_precision(seas, torch, wr, code, Vd, K, W, dist, device, stream, peak)
            variants[name] = {"value": wr.N * K * world / (r2["total_ms"] / 1e3), "unit": METRIC, "dtype": dtype,
                              "ms_per_step": r2["total_ms"] / K, "p50_ms": float(np.percentile(r2["per"], 50)),
                              "p99_ms": float(np.percentile(r2["per"], 99)), "rel_l2_vs_oracle": err_of(tau2),
                              "rel_l2_vs_headline": (tau2 - tau).norm().item() / tau.norm().item(),
                              "bytes_interaction": r2["stats"]["bytes_interaction"],
                              "roofline": {k: r2["roofline"][k] for k in (
                                  "bound", "achieved", "peak", "unit", "frac", "mean_launch_ms")}}
            s2.close()

    # batched ensemble: 8 scenarios (independent seeded histories, scenario 0 = the headline's) share one operator;
    # one persistent interaction kernel per step serves all 8 with each operator byte read once
    batched = {}
    if not args.no_batched:
        B = 8
        V8 = np.stack([wr.slip_rate(b, 0, K) for b in range(B)], axis=1).reshape(K, B * wr.N)
        V8d = torch.from_numpy(V8).to(device)
        del V8
        for name in ("bf16", "fp64"):
            code, dtype = PRECISIONS[name]
            r3, tau3, s3 = run_precision(seas, torch, wr, code, V8d, K, W, dist, device, stream, peak, batch=B)
            t0 = tau3[:, : wr.N]
            batched[name] = {"value": B * wr.N * K * world / (r3["total_ms"] / 1e3), "unit": METRIC, "batch": B,
                             "dtype": dtype, "ms_per_step": r3["total_ms"] / K,
                             "p50_ms": float(np.percentile(r3["per"], 50)),
                             "p99_ms": float(np.percentile(r3["per"], 99)),
                             "rel_l2_member0_vs_headline": (t0 - tau).norm().item() / tau.norm().item(),
                             "roofline": {k: r3["roofline"][k] for k in (
                                 "bound", "achieved", "peak", "unit", "frac", "mean_launch_ms")}}
            s3.close()
            del tau3
        del V8d

    # the flagged static tail (elastostatic response of the history the windows drop) on the headline operator
    tail = None
    if not args.no_tail:
        r4, tau4, s4 = run_precision(seas, torch, wr, head_code, Vd, K, W, dist, device, stream, peak,
                                     flags=int(wr.hparams.get("flags", 0)) | seas.SEAS_FLAG_STATIC_TAIL)
        tv = job_rate(wr.N * K, world, r4["total_ms"] / 1e3)
        tail = {"value": tv, "unit": METRIC, "ms_per_step": r4["total_ms"] / K, "cost_vs_headline": value / tv - 1,
                "tail_share_of_tau": (tau4 - tau).norm().item() / tau.norm().item()}
        s4.close()
        del tau4

    # plain FP64 GPU path: every block dense (leaf blocks, exact windows), no compression, FP64 arithmetic
    plain = None
    if not args.no_plain:
        p = seas.Session(wr, device=local, stream=stream.cuda_stream, flags=seas.SEAS_FLAG_DENSE)
        pm, pper, ptau = timed_run(seas, torch, p, Vd, K, dist, device)
        seas.seas_scenario_check(p.scn)
        pm = max_over_ranks(dist, pm, device)
        pv = wr.N * K * world / (pm / 1e3)
        plain = {"value": pv, "unit": METRIC, "ms_per_step": pm / K, "p50_ms": float(np.percentile(pper, 50)),
                 "p99_ms": float(np.percentile(pper, 99)), "speedup": value / pv,
                 "bytes_interaction": p.stats["bytes_interaction"], "rel_l2_vs_oracle": err_of(ptau),
                 "rel_l2_tau_vs_headline": (ptau - tau).norm().item() / ptau.norm().item()}
        p.close()

    # end to end through the C ABI with host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        s2 = seas.seas_scenario_create(s.op, 1)
        Vh = torch.from_numpy(V).pin_memory().numpy()
        th = torch.zeros(wr.N, dtype=torch.float64).pin_memory().numpy()
        barrier(dist)
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        for n in range(K):
            seas.seas_push_slip_rate(s2, Vh[n])
            seas.seas_stress_step(s2, th)
        torch.cuda.synchronize(device)
        barrier(dist)
        e2e_s = max_over_ranks(dist, time.perf_counter() - t0, device)
        seas.seas_destroy_scn(s2)
        e2e = {"value": wr.N * K * world / e2e_s, "unit": METRIC, "h2d_bytes_per_step": wr.N * 8,
               "d2h_bytes_per_step": wr.N * 8}

    roofline = res["roofline"]
    roofline["traffic"] = None
    tf = os.path.join(ROOT, "profiles", "interaction_traffic.json")
    if os.path.exists(tf):
        with open(tf) as fh:
            tr = json.load(fh)
        ratio = tr.get("dram_over_algorithmic", {}).get(args.precision)
        if tr.get("kernel_version") == seas_kernel_version() and ratio is not None:
            # DRAM bytes of the captured launch over its algorithmic bytes, scaled to this run's mean launch
            roofline["traffic"] = ratio * roofline["algorithmic_bytes_per_launch"]
            roofline["traffic_source"] = tr.get("source")

    line = None
    if rank == 0:
        cpu = None
        if oracle is not None:
            cpu = {"value": args.cpu_sample / oracle[3], "unit": METRIC, "cores": 1, "kind": "oracle",
                   "sample": f"{args.cpu_sample} element-steps (receivers of fault 0 at steps spread over the run, "
                             f"all lags of all sources, NumPy FP64), {oracle[3]:.1f} s"}
        launches = res["timing"]["launches"]
        line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": K, "warmup": W,
                "ms_per_step": res["total_ms"] / K, "p50_ms": float(np.percentile(res["per"], 50)),
                "p99_ms": float(np.percentile(res["per"], 99)), "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": head_dtype, "data": "synthetic",
                "config": dict(config_of(wr, K), precision=args.precision),
                "rel_l2_vs_oracle": err, "operator": {k: stats[k] for k in (
                    "n_blocks_far", "n_blocks_near", "compression_ratio", "bytes_interaction", "mean_rank",
                    "max_rank", "build_seconds", "n_tasks")},
                "vs_plain_fp64_gpu": plain, "variants": variants, "batched": batched, "static_tail": tail, "e2e": e2e,
                "roofline": roofline,
                "cpu_baseline": cpu, "clocks": res["clocks"], "gpu_launches": int(sum(launches.values()))}
    s.close()
    if dist is not None:
        dist.destroy_process_group()
    return line


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
    w = synth.WORKLOADS[args.workload]()
    K = args.steps if args.steps is not None else w.steps
    W = max(3, args.warmup)
    if args.impl == "reference":
        line = run_reference(args, w, K, W)
    else:
        from paper_2603_00383_gb300 import build
        build.build()
        line = run_ours(args, w, K, W)
    if line is not None:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
