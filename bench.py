#!/usr/bin/env python3
"""Benchmark of the blocked Cholesky derivative path on one GB300 (or N
independent replicas under torchrun).

One step = one pass of the whole hot path on one synthetic problem:
chol_fwd(Sigma) -> L, chol_fwd_sens(L, Sigma_dot) -> L_dot and
chol_rev(L, L_bar) -> tril(Sigma_bar), with the in-place inputs restored from
pristine device copies at the start of the step.  The headline value is the
reverse pass's throughput, nominal 2 N^3 / 3 flops over its device time
(CUDA events on the launching stream), at N = 8192 on a squared-exponential
covariance (ell 0.3 on [0,1]^3, jitter 1e-4).

  python bench.py [--gpus N] [--steps K] [--warmup W]       # our CUDA path
  python bench.py --impl reference ...                        # the CPU oracle

Prints one JSON line (rank 0).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "chol_rev TFLOP/s @N=8192 (FP64 vs mixed, err vs FP64); served fwd+rev p99 latency"
UNIT = "TFLOP/s"
# FP64 is a plain-ALU (DFMA) path on GB300: 152 SMs x 2 DFMA/clk x 2 flop x 2.070 GHz.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12
# ncu, k_gemm_f64<N,T> (64 x 64 tiles) in the FP64 step at N=4096: 28.0 MB of DRAM traffic
# (dram__bytes_read.sum + dram__bytes_write.sum) per launch of 0.734 GFLOP on average
GEMM_NT_DRAM_BYTES_PER_FLOP = 28.0e6 / 0.734e9
SE_SEED = 2


def _bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except (OSError, ValueError, KeyError):
        return 1900.0  # measured fallback for GB300


BF16_PEAK_TFLOPS = _bf16_peak()


def flops_fwd(n):
    return n ** 3 / 3.0


def flops_rev(n):
    return 2.0 * n ** 3 / 3.0


def flops_sens(n):
    return 2.0 * n ** 3 / 3.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--nb", type=int, default=0)
    ap.add_argument("--diag", default="auto", choices=["auto", "level2", "symbolic"])
    ap.add_argument("--cpu-n", type=int, default=6144, help="oracle sample size for cpu_baseline")
    ap.add_argument("--ref-n", type=int, default=4096, help="oracle sample size per reference step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-dual", action="store_true", help="skip the one-loop chol_fwd_and_sens leg")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-sweep", action="store_true", help="skip the FP64 block-size sweep (N 4096/8192, nb 64-256)")
    ap.add_argument("--no-peak", action="store_true", help="skip the FP64 peak probes")
    ap.add_argument("--serve-seconds", type=float, default=10.0, help="length of the served Poisson stream")
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-lanes", type=int, default=2)
    ap.add_argument("--serve-sustained-rate", type=float, default=250.0,
                    help="a second, sustainable arrival rate (about 80%% of measured capacity)")
    ap.add_argument("--profile-pass", default=None, choices=["fwd", "sens", "rev", "fwd_and_sens"],
                    help="for profilers: run one pass of this operation on the --n workload and exit "
                         "(no timing, no JSON line); the factor it needs is computed first in FP64")
    ap.add_argument("--prec", default="fp64", choices=["fp64", "bf16x3", "bf16x6", "fixed4"],
                    help="precision of the --profile-pass operation")
    ap.add_argument("--profile-gemm", default=None, metavar="M,N,K",
                    help="for profilers: run the --prec tensor-core product (bf16x3, bf16x6 or fixed4) of "
                         "random M x K and N x K operands three times and exit (no JSON line)")
    ap.add_argument("--timeline", action="store_true",
                    help="with --profile-pass: warm up, then print the recorded pass's launch timeline")
    return ap.parse_args()


def profile_gemm(args):
    """Three calls of one tensor-core product, for a profiler to capture the last."""
    import torch
    from paper_1602_07527_gb300 import native as nat
    M, N, K = (int(v) for v in args.profile_gemm.split(","))
    prec = args.prec if args.prec != "fp64" else "fixed4"
    dev = torch.device("cuda", 0)
    g = torch.Generator(device=dev).manual_seed(0)
    A = torch.randn(M, K, generator=g, device=dev, dtype=torch.float64)
    B = torch.randn(N, K, generator=g, device=dev, dtype=torch.float64)
    C = torch.zeros(M, N, dtype=torch.float64, device=dev)
    for _ in range(3):
        nat.mixed_gemm_debug(A, B, C, prec=prec)
    torch.cuda.synchronize()
    print(f"profile product done: {prec} M={M} N={N} K={K}", file=sys.stderr)
    return 0


def profile_pass(args):
    """One pass of one operation, for a profiler to capture: the FP64 SE workload
    for --prec fp64, the Matern-5/2 workload for the split-BF16 precisions.
    With --timeline, a warm-up pass first, then the library's own launch
    timeline of the recorded pass (kernel, stream, start and end) on stdout."""
    import torch
    import paper_1602_07527_gb300 as cd
    from paper_1602_07527_gb300 import workloads as W

    dev = torch.device("cuda", 0)
    n = args.n
    if args.prec == "fp64":
        S, Lb = W.large_se_case(n, SE_SEED)
        seed = SE_SEED
    else:
        S, Lb = W.mixed_matern_case(n, 3)
        seed = 3
    A0 = torch.tensor(np.tril(S), device=dev)
    del S
    op = args.profile_pass
    if op in ("fwd", "fwd_and_sens"):
        Ad0 = torch.tensor(np.tril(W.sigma_dot(n, seed)), device=dev) if op == "fwd_and_sens" else None
        L = None
    else:
        L = A0.clone()
        if int(cd.chol_fwd(L).item()) != 0:  # the FP64 factor the derivative pass takes as input
            raise RuntimeError("factorisation reported a non-positive pivot")
        X0 = torch.tensor(Lb if op == "rev" else np.tril(W.sigma_dot(n, seed)), device=dev)

    def run():
        if op == "fwd":
            A = A0.clone()
            return cd.chol_fwd(A, nb=args.nb, prec=args.prec)
        if op == "fwd_and_sens":
            A, Ad = A0.clone(), Ad0.clone()
            return cd.chol_fwd_and_sens(A, Ad, nb=args.nb, prec=args.prec, diag=args.diag)
        X = X0.clone()
        if op == "rev":
            cd.chol_rev(L, X, nb=args.nb, prec=args.prec, diag=args.diag)
        else:
            cd.chol_fwd_sens(L, X, nb=args.nb, prec=args.prec, diag=args.diag)
        return None

    if args.timeline:
        run()
        torch.cuda.synchronize()
        cd.profile_read(dev)
        cd.profile_enable(True, dev)
    info = run()
    torch.cuda.synchronize()
    if info is not None and int(info.item()) != 0:
        raise RuntimeError("factorisation reported a non-positive pivot")
    if args.timeline:
        tl = cd.profile_timeline(dev)
        cd.profile_read(dev)
        cd.profile_enable(False, dev)
        print(f"# launch timeline: {op} {args.prec} N={n} nb={args.nb or 'default'}: {len(tl)} launches, "
              f"span {tl[-1]['end_ms'] if tl else 0.0:.3f} ms (per-launch CUDA events; stream 1 = side stream)")
        print("stream  kernel                                   start_us    end_us   dur_us")
        for r in tl:
            print(f"{r['stream']:6d}  {r['name']:38s} {1e3 * r['start_ms']:9.1f} {1e3 * r['end_ms']:9.1f} "
                  f"{1e3 * (r['end_ms'] - r['start_ms']):8.1f}")
    print(f"profile pass done: {op} {args.prec} N={n}", file=sys.stderr)
    return 0


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only: no data-path collective)
# ---------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Dist:
    def __init__(self, backend):
        import torch
        import torch.distributed as dist
        self.ws, self.rank, self.local = dist_env()
        self.dist = dist if self.ws > 1 else None
        self.torch = torch
        if self.dist:
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            dist.init_process_group(backend)

    def barrier(self):
        if self.dist:
            self.dist.barrier()

    def max(self, x):
        if not self.dist:
            return x
        t = self.torch.tensor([float(x)], device="cuda" if self.torch.cuda.is_available() else "cpu")
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.dist:
            self.dist.destroy_process_group()


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline leg and the reference arm)
# ---------------------------------------------------------------------------
def oracle_rev_sample(n):
    import oracle
    from paper_1602_07527_gb300 import workloads as W
    S, Lb = W.large_se_case(n, SE_SEED)
    L, info = oracle.chol_unblocked(S)
    if info:
        raise RuntimeError(f"oracle factorisation failed at column {info}")
    t = time.perf_counter()
    oracle.chol_unblocked_rev(L, Lb)
    dt = time.perf_counter() - t
    return dt, oracle.num_threads()


def cpu_baseline(n):
    dt, cores = oracle_rev_sample(n)
    return {"value": flops_rev(n) / dt / 1e12, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": (f"one oracle chol_unblocked_rev (plain C, OpenMP rows) at N={n} on the same SE "
                       f"recipe (seed {SE_SEED}), {dt:.2f} s; throughput = 2N^3/3 / time")}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    n = args.ref_n
    for _ in range(args.warmup):
        oracle_rev_sample(n)
    times, cores = [], 1
    for _ in range(args.steps):
        dt, cores = oracle_rev_sample(n)
        times.append(dt)
    tot = sum(times)
    value = flops_rev(n) * args.steps / tot / 1e12
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "impl": "reference",
        # the metric's workload (ours_config) sampled at N = ref_n: the oracle's
        # O(N^3) scalar loop would take minutes per step at the full N
        "config": dict(ours_config(args), workload=(
            f"chol_rev FP64, SE covariance ell 0.3 on [0,1]^3 + 1e-4 I (seed {SE_SEED}): oracle sample at "
            f"N={n} per step (our arm's N={args.n}); throughput scales the sample by 2N^3/3"), n=n,
            sample_of_n=args.n),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"each step: one oracle chol_unblocked_rev at N={n} (same SE recipe)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def ours_config(args):
    return {"workload": f"chol_rev FP64 N={args.n}, SE covariance ell 0.3 on [0,1]^3 + 1e-4 I (seed {SE_SEED})",
            "n": args.n, "nb": args.nb or "default", "diag": args.diag,
            "step": "chol_fwd -> chol_fwd_sens -> chol_rev on one N x N problem",
            "l2": "inputs exceed L2 (512 MiB per FP64 matrix at N=8192); no flush",
            "parallelism": "replicas (one independent problem per GPU)"}


def fp64_peak_leg(dev):
    """The FP64 pipe's rate on this GPU: register-only DFMA chains (the
    instruction of the library's FP64 products) and the FP64 matrix
    instruction (mma.sync m8n8k4), each timed with CUDA events."""
    import torch
    from paper_1602_07527_gb300 import native as nat
    out = {}
    stream = torch.cuda.current_stream(dev)
    for kind in ("dfma", "dmma"):
        nat.fp64_probe(kind, 20000, dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fl = nat.fp64_probe(kind, 400000, dev)
        e1.record(stream)
        torch.cuda.synchronize()
        out[kind + "_tflops"] = fl / (e0.elapsed_time(e1) * 1e-3) / 1e12
    out["derived_dfma_tflops"] = FP64_PEAK_TFLOPS
    out["how"] = ("4 CTAs x 256 threads per SM, register operands only: a 4 x 2 outer product of FMAs a "
                  "thread (dfma) or 4 chains of mma.sync m8n8k4 f64 a thread (dmma); CUDA events")
    return out


def nb_sweep_leg(args, dev):
    """Block size sweep of the large FP64 configuration: SE covariance (ell 0.3
    on [0,1]^3 + 1e-4 I), N in {4096, 8192}, nb in {64, 128, 256}; median of
    three CUDA-event-timed calls after one warm-up, inputs restored outside the
    timed region."""
    import torch
    import paper_1602_07527_gb300 as cd
    from paper_1602_07527_gb300 import workloads as W
    stream = torch.cuda.current_stream(dev)
    rows = []
    for n in (4096, 8192):
        S, Lb = W.large_se_case(n, SE_SEED)
        S0 = torch.tensor(np.tril(S), device=dev)
        Lb0 = torch.tensor(Lb, device=dev)
        del S, Lb
        L = S0.clone()
        cd.chol_fwd(L)
        X = torch.empty_like(S0)
        for nb in (64, 128, 256):
            t = {}
            for op in ("chol_fwd", "chol_rev"):
                ms = []
                for r in range(4):
                    X.copy_(S0 if op == "chol_fwd" else Lb0)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    if op == "chol_fwd":
                        cd.chol_fwd(X, nb=nb)
                    else:
                        cd.chol_rev(L, X, nb=nb)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    if r:
                        ms.append(e0.elapsed_time(e1))
                m = statistics.median(ms)
                fl = flops_fwd(n) if op == "chol_fwd" else flops_rev(n)
                t[op] = {"ms": m, "tflops": fl / (m * 1e-3) / 1e12}
            rows.append({"n": n, "nb": nb, **t})
        del S0, Lb0, L, X
        torch.cuda.empty_cache()
    return rows


# ---------------------------------------------------------------------------
# our CUDA path
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch
    import paper_1602_07527_gb300 as cd
    from paper_1602_07527_gb300 import workloads as W

    d = Dist("nccl")
    torch.cuda.set_device(d.local)
    dev = torch.device("cuda", d.local)
    n, nb = args.n, args.nb

    S, Lb = W.large_se_case(n, SE_SEED)
    Sd = W.sigma_dot(n, SE_SEED)
    S0 = torch.tensor(np.tril(S), device=dev)
    Lb0 = torch.tensor(Lb, device=dev)
    Sd0 = torch.tensor(np.tril(Sd), device=dev)
    del S, Sd
    A = torch.empty_like(S0)
    Ab = torch.empty_like(Lb0)
    Ad = torch.empty_like(Sd0)
    stream = torch.cuda.current_stream(dev)
    cd.reserve(cd.workspace_size(n, nb), dev)

    def step(prec="fp64"):
        A.copy_(S0)
        Ab.copy_(Lb0)
        Ad.copy_(Sd0)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        info = cd.chol_fwd(A, nb=nb, prec=prec)
        ev[1].record(stream)
        cd.chol_fwd_sens(A, Ad, nb=nb, prec=prec, diag=args.diag)
        ev[2].record(stream)
        cd.chol_rev(A, Ab, nb=nb, prec=prec, diag=args.diag)
        ev[3].record(stream)
        return ev, info

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    cd.profile_read(dev)  # discard warm-up records
    clocks = ClockSampler(d.local)
    d.barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = cd.launch_count(dev)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    evs = []
    for _ in range(args.steps):
        evs.append(step())
    t1.record(stream)
    torch.cuda.synchronize()
    d.barrier()
    clock_info = clocks.stop()
    launches = cd.launch_count(dev) - launches0
    total_ms = d.max(t0.elapsed_time(t1))
    # the per-kernel profile (an event pair around every launch) from one more
    # step after the timed ones, so that its events do not slow the timed steps
    cd.profile_enable(True, dev)
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    step()
    p1.record(stream)
    torch.cuda.synchronize()
    kstats = cd.profile_read(dev)
    cd.profile_enable(False, dev)
    prof_ms = p0.elapsed_time(p1)
    op_ms = {"chol_fwd": [], "chol_fwd_sens": [], "chol_rev": []}
    for ev, info in evs:
        op_ms["chol_fwd"].append(ev[0].elapsed_time(ev[1]))
        op_ms["chol_fwd_sens"].append(ev[1].elapsed_time(ev[2]))
        op_ms["chol_rev"].append(ev[2].elapsed_time(ev[3]))
        if int(info.item()) != 0:
            raise RuntimeError("factorisation reported a non-positive pivot")
    rev_ms = d.max(statistics.median(op_ms["chol_rev"]))
    value = d.ws * flops_rev(n) / (rev_ms * 1e-3) / 1e12
    ops = {k: {"ms_median": statistics.median(v),
               "tflops": {"chol_fwd": flops_fwd, "chol_fwd_sens": flops_sens, "chol_rev": flops_rev}[k](n)
               / (statistics.median(v) * 1e-3) / 1e12} for k, v in op_ms.items()}

    # the one-loop factorisation + forward sensitivity (Sec. 4.1-4.2) on the
    # same inputs, against the two separate calls of the step above
    def dual_step(prec="fp64"):
        A.copy_(S0)
        Ad.copy_(Sd0)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        e[0].record(stream)
        info = cd.chol_fwd_and_sens(A, Ad, nb=nb, prec=prec, diag=args.diag)
        e[1].record(stream)
        return e, info

    def time_dual(prec="fp64"):
        for _ in range(max(1, args.warmup - 1)):
            dual_step(prec)
        evs_d = [dual_step(prec) for _ in range(args.steps)]
        torch.cuda.synchronize()
        if any(int(i.item()) != 0 for _, i in evs_d):
            raise RuntimeError("factorisation reported a non-positive pivot")
        return statistics.median(e[0].elapsed_time(e[1]) for e, _ in evs_d)

    dual = None
    if not args.no_dual:
        dm = time_dual()
        sep = ops["chol_fwd"]["ms_median"] + ops["chol_fwd_sens"]["ms_median"]
        dual = {"ms_median": dm, "tflops": (flops_fwd(n) + flops_sens(n)) / (dm * 1e-3) / 1e12,
                "separate_ms": sep, "speedup_vs_separate": sep / dm}

    peak = None if args.no_peak else fp64_peak_leg(dev)
    fp64_peak = peak["dfma_tflops"] if peak else FP64_PEAK_TFLOPS
    # executed work of the profiled step (the library's per-launch algorithmic
    # flops, all terms) beside the nominal N^3/3 + 2 N^3/3 + 2 N^3/3
    flops_exec = {"executed_step": sum(k["flops"] for k in kstats),
                  "nominal_step": flops_fwd(n) + flops_sens(n) + flops_rev(n)}
    # roofline of the dominant kernel (largest total device time in the profiled step)
    dom = kstats[0] if kstats else None
    roofline = None
    if dom:
        achieved = dom["flops"] / (dom["ms"] * 1e-3) / 1e12 if dom["ms"] > 0 else 0.0
        # DRAM bytes per launch of the FP64 N,T product from ncu (dram__bytes_read.sum +
        # dram__bytes_write.sum) at N=4096, scaled to this launch's average work
        traffic = None
        if dom["name"] == "gemm_f64<N,T>" and dom["launches"] > 0:
            traffic = GEMM_NT_DRAM_BYTES_PER_FLOP * dom["flops"] / dom["launches"]
        roofline = {"bound": "alu", "kernel": dom["name"], "achieved": achieved, "peak": fp64_peak,
                    "unit": "TFLOP/s", "frac": achieved / fp64_peak, "traffic": traffic,
                    "traffic_source": ("ncu at N=4096 (two launches: 28.0 MB in 0.734 GFLOP), scaled by the "
                                       "launch's flops" if traffic is not None else None),
                    "peak_source": ("measured in this run: DFMA chains on every SM (fp64_peak.dfma_tflops), "
                                    "of measured" if peak else
                                    "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.070 GHz (FP64 pipe)"),
                    "frac_of_derived_pipe": achieved / FP64_PEAK_TFLOPS,
                    "launches": dom["launches"], "ms_per_launch": dom["ms"] / max(1, dom["launches"]),
                    "share_of_profiled_step": dom["ms"] / prof_ms,
                    "measured_over": "one profiled step after the timed steps (CUDA events on the kernel's stream)"}
    kernels = [{"name": k["name"], "launches": k["launches"], "ms": round(k["ms"], 3),
                "share": k["ms"] / prof_ms,
                "tflops": (k["flops"] / (k["ms"] * 1e-3) / 1e12) if k["ms"] > 0 else 0.0}
               for k in kstats[:8]]

    # end to end through the public call with host buffers (pinned), rev only
    e2e = None
    if not args.no_e2e:
        Lh = A.cpu().pin_memory()
        Lbh = Lb0.cpu().pin_memory()
        outh = torch.empty_like(Lbh).pin_memory()
        Ld = torch.empty_like(A)
        Abd = torch.empty_like(Ab)

        def e2e_step():
            Ld.copy_(Lh, non_blocking=True)
            Abd.copy_(Lbh, non_blocking=True)
            cd.chol_rev(Ld, Abd, nb=nb)
            outh.copy_(Abd, non_blocking=True)

        e2e_step()
        torch.cuda.synchronize()
        ks = max(1, args.steps)
        d.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(ks):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = d.max(e0.elapsed_time(e1) / ks)
        e2e = {"value": d.ws * flops_rev(n) / (e2e_ms * 1e-3) / 1e12, "unit": UNIT,
               "h2d_bytes_per_step": 2 * n * n * 8, "d2h_bytes_per_step": n * n * 8,
               "ms_per_step": e2e_ms, "path": "pinned host L, L_bar -> device -> cd_chol_rev -> host Sigma_bar"}

    # mixed precision on the same inputs: split-BF16 products on the tensor
    # cores, diagonal tiles in FP64; errors against this run's FP64 results
    mixed = None
    if not args.no_mixed:
        # the mixed-precision workload: Matern-5/2 (ell 0.2) on [0,1]^4 + 1e-3 I,
        # condition number below 1e6; FP64 reference computed here on the same inputs
        Sm, Lbm = W.mixed_matern_case(n, 3)
        S0.copy_(torch.tensor(np.tril(Sm)))
        Lb0.copy_(torch.tensor(Lbm))
        Sd0.copy_(torch.tensor(np.tril(W.sigma_dot(n, 3))))
        del Sm, Lbm
        step("fp64")
        torch.cuda.synchronize()
        ref_L, ref_Ld, ref_Sb = A.clone(), Ad.clone(), Ab.clone()
        Lexact = A.clone()
        mixed = {"workload": f"Matern-5/2 ell 0.2 on [0,1]^4 + 1e-3 I, N={n} (seed 3); errors vs the FP64 path"}
        for prec in ("fixed4", "bf16x6", "bf16x3"):
            for _ in range(max(1, args.warmup - 1)):
                step(prec)
            torch.cuda.synchronize()
            # timed without per-launch profiling events; one profiled step after
            mevs = [step(prec) for _ in range(args.steps)]
            torch.cuda.synchronize()
            cd.profile_read(dev)
            cd.profile_enable(True, dev)
            step(prec)
            torch.cuda.synchronize()
            mk = cd.profile_read(dev)
            cd.profile_enable(False, dev)
            mrev = statistics.median(ev[2].elapsed_time(ev[3]) for ev, _ in mevs)
            mfwd = statistics.median(ev[0].elapsed_time(ev[1]) for ev, _ in mevs)
            msens = statistics.median(ev[1].elapsed_time(ev[2]) for ev, _ in mevs)
            rel = lambda x, r: float(torch.linalg.norm(torch.tril(x - r)) / torch.linalg.norm(torch.tril(r)))
            e = {"L": rel(A, ref_L), "L_dot": rel(Ad, ref_Ld), "Sigma_bar": rel(Ab, ref_Sb)}
            # reverse pass alone, given the FP64 factor
            Ab.copy_(Lb0)
            cd.chol_rev(Lexact, Ab, nb=nb, prec=prec)
            e["Sigma_bar_given_fp64_L"] = rel(Ab, ref_Sb)
            Ad.copy_(Sd0)
            cd.chol_fwd_sens(Lexact, Ad, nb=nb, prec=prec)
            e["L_dot_given_fp64_L"] = rel(Ad, ref_Ld)
            e["max"] = max(e.values())
            if not args.no_dual:
                dms = time_dual(prec)
                entry_dual = {"ms": dms, "separate_ms": mfwd + msens, "speedup_vs_separate": (mfwd + msens) / dms,
                              "rel_err_vs_fp64": {"L": rel(A, ref_L), "L_dot": rel(Ad, ref_Ld)}}
            # the tensor-core kernel with the most work (the bulk product); the chain's small
            # products can take longer in total while doing little of the work
            tk = max((k for k in mk if k["name"].startswith(("mgemm", "fgemm"))), key=lambda k: k["flops"],
                     default=None)
            entry = {"chol_rev_tflops": d.ws * flops_rev(n) / (d.max(mrev) * 1e-3) / 1e12,
                     "chol_fwd_tflops": flops_fwd(n) / (mfwd * 1e-3) / 1e12,
                     "chol_fwd_sens_tflops": flops_sens(n) / (msens * 1e-3) / 1e12,
                     "ms": {"chol_fwd": mfwd, "chol_fwd_sens": msens, "chol_rev": mrev},
                     "rel_err_vs_fp64": e,
                     "speedup_rev_vs_fp64": rev_ms / mrev,
                     "kernels": [{"name": k["name"], "launches": k["launches"], "ms": round(k["ms"], 3)}
                                 for k in mk[:6]]}
            if tk:
                ach = tk["flops"] / (tk["ms"] * 1e-3) / 1e12
                entry["tensor_roofline"] = {"bound": "tensor", "kernel": tk["name"], "achieved": ach,
                                            "peak": BF16_PEAK_TFLOPS, "unit": "TFLOP/s",
                                            "frac": ach / BF16_PEAK_TFLOPS,
                                            "peak_source": "MEASURED_PEAKS.json bf16_tflops (cuBLAS burst)",
                                            "selection": "the tensor-core kernel with the most work in the "
                                                         "profiled step"}
            if not args.no_dual:
                entry["fwd_and_sens"] = entry_dual
            mixed[prec] = entry

    sweep = None
    if not args.no_sweep:
        del A, Ab, Ad
        torch.cuda.empty_cache()
        sweep = nb_sweep_leg(args, dev)
        A, Ab, Ad = torch.empty_like(S0), torch.empty_like(Lb0), torch.empty_like(Sd0)

    serving = None
    if not args.no_serving:
        del A, Ab, Ad, S0, Lb0, Sd0
        torch.cuda.empty_cache()
        serving = serve_bench(args, dev)

    cpu = None
    if d.rank == 0 and d.ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.cpu_n)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": d.ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic: SE covariance (ell 0.3, points U[0,1]^3, jitter 1e-4), L_bar and Sigma_dot iid N(0,1)",
        "config": ours_config(args), "ops": ops, "roofline": roofline, "kernels": kernels,
        "fwd_and_sens": dual, "mixed": mixed, "serving": serving, "nb_sweep": sweep, "fp64_peak": peak,
        "flops": flops_exec,
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clock_info,
        "step_tflops": d.ws * (flops_fwd(n) + flops_sens(n) + flops_rev(n)) / (total_ms / args.steps * 1e-3) / 1e12,
    }
    if d.rank == 0:
        print(json.dumps(line), flush=True)
    d.close()
    return 0


def serve_bench(args, dev):
    """Served fwd+rev: Poisson arrivals, N log-uniform in [32, 4096], half FP64
    and half split-BF16 (x6), 40 GB HBM budget; p50/p99 latency and solves/s,
    next to a sample of the same requests run alone on the idle GPU."""
    import torch
    from paper_1602_07527_gb300 import serving as sv
    from paper_1602_07527_gb300 import workloads as W
    stream = W.serving_stream(seed=5, rate=args.serve_rate, duration=args.serve_seconds)
    reqs = sv.requests_from_stream(stream, mixed_prec="bf16x6")
    # the full stream's inputs (about 28 MB a request) do not all fit in HBM at
    # once: each request's inputs are drawn on the device from its seed when its
    # batch is launched (about 0.1 ms of device time against a solve of 1-60 ms)
    prepared = sum(sv.request_bytes(r.n, r.prec) for r in reqs) <= 100e9
    if prepared:
        sv.prepare(reqs, dev)  # payloads resident in HBM before the replay starts
    # warm the lanes (workspace growth, first-launch costs) on a few requests
    warm = sv.Server(dev, mem_cap=40e9, lanes_per_prec=args.serve_lanes, precisions=("fp64", "bf16x6"))
    warm.run(sv.requests_from_stream(W.serving_stream(seed=6, rate=2000.0, duration=0.01)), realtime=False)
    torch.cuda.synchronize()
    server = warm
    t0 = time.perf_counter()
    done = server.run(reqs, realtime=True)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    offered = sv.summarize(done, wall)
    by_prec = {p: sv.summarize([r for r in done if r.prec == p], wall) for p in ("fp64", "bf16x6")}
    # the same kinds of requests alone: a sample of 1000, one at a time on the idle GPU
    rng = np.random.default_rng(7)
    sample = [reqs[i] for i in sorted(rng.choice(len(reqs), size=min(1000, len(reqs)), replace=False))]
    alone = []
    for r in sample:
        r.payload = sv.build_inputs(r, dev)
        torch.cuda.synchronize()
        t = time.perf_counter()
        sv.solve_alone(r, dev)
        torch.cuda.synchronize()
        alone.append(time.perf_counter() - t)
        r.payload = None
    served_sample = [r.t_done - r.t_admit for r in done if r.rid in {q.rid for q in sample}]
    for r in reqs:
        r.payload = None
    torch.cuda.empty_cache()
    # the same mix at a rate the GPU sustains: queueing no longer dominates
    sus_stream = W.serving_stream(seed=8, rate=args.serve_sustained_rate, duration=args.serve_seconds)
    sus_reqs = sv.requests_from_stream(sus_stream, mixed_prec="bf16x6")
    sv.prepare(sus_reqs, dev)
    t1 = time.perf_counter()
    sus_done = server.run(sus_reqs, realtime=True)
    torch.cuda.synchronize()
    sus_wall = time.perf_counter() - t1
    sustained = sv.summarize(sus_done, sus_wall)
    sustained["rate"] = args.serve_sustained_rate
    sustained["by_precision"] = {p: sv.summarize([r for r in sus_done if r.prec == p], sus_wall)
                                 for p in ("fp64", "bf16x6")}
    server.close()
    mean_n3 = float(np.mean([r.n ** 3 for r in reqs]))
    return {"stream": (f"Poisson {args.serve_rate:g} req/s for {args.serve_seconds:g} s, N log-uniform [32, 4096], "
                       + ("payloads resident in HBM before the replay, " if prepared else
                          "payloads drawn on the device from each request's seed at launch, ") +
                       f"50/50 FP64 / split-BF16 x6, SE ell 0.3 on [0,1]^3 + {sv.SE_JITTER:g} I, 40 GB budget, "
                       f"{args.serve_lanes} lanes per precision"),
            "offered_tflops": args.serve_rate * mean_n3 / 1e12,
            "served": offered, "served_by_precision": by_prec, "sustained": sustained,
            "peak_bytes": server.peak_bytes, "lane_workspace_bytes": server.ws_total,
            "admission": "HBM budget = the lanes' reserved workspaces + the buffers of requests in flight",
            "host_launch_s": server.host_launch_s, "host_phase_s": server.host_phase_s,
            "alone_sample": {"requests": len(alone), "p50_ms": 1e3 * sv.percentile(alone, 50),
                             "p99_ms": 1e3 * sv.percentile(alone, 99),
                             "solves_per_s": len(alone) / sum(alone),
                             "served_service_p50_ms_same_requests": 1e3 * sv.percentile(served_sample, 50)}}


def main():
    args = parse()
    if args.profile_gemm:
        return profile_gemm(args)
    if args.profile_pass:
        return profile_pass(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
