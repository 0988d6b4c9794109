"""Benchmark of the Wilson-Dirac hot path on GB300.

A step is one full CG solve of D x = b on the normal equations to a true FP64
residual of 1e-10 (section 2.2), on seeded synthetic inputs:

  c3 (default)  32^3 x 64, smoothed links exp(i 0.4 H), kappa = 0.124, Gaussian
                source, plain FP64 CGNR (the largest single-GPU workload)
  c2            16^4, Haar-random SU(3) links, kappa = 0.12, Gaussian source
  c1            4^4, same recipe
  c4            24^3 x 48, Haar links, kappa = 0.12, the 12 spin-colour point
                sources solved together (multi-RHS CG)
  (--inner f32|f16|df32 runs the step with that inner precision instead)

value = GFLOP/s of the solve at 1320 flop per site per Dslash application,
counting the operator applications the solve performs (2 per iteration, D^dag b
in the setup, the two of the final FP64 check; a zero start vector skips the
setup's D x0 pair).  The roofline object describes the plain Dslash kernel of
the step's precision on the same lattice, timed alone; for FP64 its roof is the
FP64 multiply-add rate measured in the same run (wd_measure_fp64_rate).  The
`cg` object times every solver variant on the same lattice and source (mixed
precision, even-odd, compressed inner links, the system-residual stopping rule)
against the FP64 step, and `multi_rhs` the 12 point sources of the 24^3 x 48
workload solved together against 12 sequential FP64 solves.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c3]
  python bench.py --impl reference ...   # the CPU oracle as the reference arm
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

FLOP_PER_SITE = 1320
# Algorithmic bytes per site of one Dslash (each input field read once, output
# written once): spinor in + links + spinor out.
SPINOR_BYTES = {"f64": 192, "f32": 96, "f16": 52, "df32": 192}
LINK_BYTES = {("f64", 18): 576, ("f64", 12): 384, ("f64", 8): 256, ("f32", 18): 288, ("f32", 12): 192,
              ("f32", 8): 128, ("f16", 18): 144, ("f16", 12): 96, ("f16", 8): 64, ("df32", 18): 576,
              ("df32", 12): 384, ("df32", 8): 256}
PREC_ID = {"f64": 0, "f32": 1, "f16": 2, "df32": 3}
WORKLOADS = {
    "c1": dict(dims=(4, 4, 4, 4), links="haar", kappa=0.12, nrhs=1, inner="f64", seed=1),
    "c2": dict(dims=(16, 16, 16, 16), links="haar", kappa=0.12, nrhs=1, inner="f64", seed=2),
    "c3": dict(dims=(32, 32, 32, 64), links="smoothed", kappa=0.124, nrhs=1, inner="f64", seed=6),
    "c4": dict(dims=(24, 24, 24, 48), links="haar", kappa=0.12, nrhs=12, inner="f64", seed=7),
}
L2_FLUSH_BYTES = 512 << 20


def dslash_bytes(prec: str, recon: int) -> int:
    return 2 * SPINOR_BYTES[prec] + LINK_BYTES[(prec, recon)]


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": d.get("hbm_gbs"), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


# Nominal FP64 rate of a GB300: 152 SMs x 2 FP64 FMAs per clock x 2 flop x 2.07 GHz.
FP64_NOMINAL_GFLOPS = 152 * 2 * 2 * 2.07


# the sources that define the plain Dslash kernel (the one the roofline object reports)
DSLASH_SOURCES = ("df32.cuh", "wd_internal.cuh", "dslash.cuh", "dslash_apply.cu")


def csrc_hash(read=None) -> str:
    """Hash of the Dslash kernel sources; `read(name)` may supply another version of them."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1810_04201_gb300", "csrc")
    for n in DSLASH_SOURCES:
        if read is None:
            with open(os.path.join(d, n), "rb") as f:
                data = f.read()
        else:
            data = read(n)
        h.update(n.encode() + data)
    return h.hexdigest()[:16]


def recorded_traffic(kernel_key: str):
    """DRAM bytes per launch recorded by ncu for this kernel, if the sources are unchanged."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(kernel_key)
    if not e or e.get("csrc_hash") != csrc_hash():
        return None
    return e.get("bytes_per_launch")


class NvmlClockSampler:
    """SM clock and clock-event reasons read through NVML (read-only queries) every
    10 ms while the timed region runs.  Raises on start if NVML is not usable."""

    # clock-event reason bits of NVML's public header
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}

    def __init__(self, cuda_index=0, period_s=0.01):
        import ctypes
        self.ct = ctypes
        self.period = period_s
        self.nvml = ctypes.CDLL("libnvidia-ml.so.1")
        if self.nvml.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.h = ctypes.c_void_p()
        ok = False
        try:
            import torch
            uuid = "GPU-" + str(torch.cuda.get_device_properties(cuda_index).uuid)
            ok = self.nvml.nvmlDeviceGetHandleByUUID(uuid.encode(), ctypes.byref(self.h)) == 0
        except Exception:
            ok = False
        if not ok and self.nvml.nvmlDeviceGetHandleByIndex_v2(cuda_index, ctypes.byref(self.h)) != 0:
            raise RuntimeError("no NVML handle")
        self.get_reasons = getattr(self.nvml, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.nvml.nvmlDeviceGetCurrentClocksThrottleReasons
        self.samples, self.reasons, self.stop_flag = [], 0, False

    def _sm_clock(self, fn):
        v = self.ct.c_uint()
        return v.value if fn(self.h, 1, self.ct.byref(v)) == 0 else None  # 1 = NVML_CLOCK_SM

    def _run(self):
        r = self.ct.c_ulonglong()
        while not self.stop_flag:
            c = self._sm_clock(self.nvml.nvmlDeviceGetClockInfo)
            if c is not None:
                self.samples.append(c)
            if self.get_reasons(self.h, self.ct.byref(r)) == 0:
                self.reasons |= r.value
            time.sleep(self.period)

    def start(self):
        self.thread = threading.Thread(target=self._run, daemon=True)
        self.thread.start()

    def stop(self):
        self.stop_flag = True
        self.thread.join(timeout=5)
        smax = self._sm_clock(self.nvml.nvmlDeviceGetMaxClockInfo)
        return {"sm_mhz": statistics.median(self.samples) if self.samples else None, "sm_max_mhz": smax,
                "reasons": sorted(n for b, n in self.REASONS.items() if self.reasons & b),
                "samples": len(self.samples), "source": "nvml, 10 ms"}


def clock_sampler(index=0):
    try:
        return NvmlClockSampler(index)
    except Exception:
        return ClockSampler(index)


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples taken while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.out = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.out.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm), "source": "nvidia-smi, 200 ms"}


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The slowest rank's time: every rank gets the maximum of x over the job."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(flops_per_rank_step: float, step_ms: float, world: int) -> float:
    """Whole-job GFLOP/s: every rank solves its own lattice (replicas), timed by the slowest."""
    return world * flops_per_rank_step / (step_ms * 1e-3) / 1e9


def make_inputs(w, rank):
    from paper_1810_04201_gb300 import gen
    seed = w["seed"] + 1000 * rank
    dims = w["dims"]
    if w["links"] == "haar":
        U = gen.haar_links(dims, seed)
    else:
        U = gen.smoothed_links(dims, seed, eps=0.4)
    if w["nrhs"] == 12:
        b = gen.propagator_sources(dims)
    else:
        b = gen.gaussian_source(dims, seed)
    return U, b


def cpu_baseline(w, U, b, budget_s=20.0, one_core=True):
    """The oracle, as it stands, on a bounded sample of the same solve (a fixed number
    of CG iterations on the same lattice and source), on all host cores; with one_core,
    also the oracle operator's rate on one core, measured on a bounded sample of sites."""
    import oracle
    dims = w["dims"]
    V = int(np.prod(dims))
    b1 = b[0] if b.ndim == 4 else b
    threads = os.cpu_count() or 1
    oracle.set_threads(threads)
    t0 = time.perf_counter()
    oracle.apply_D(U, b1, w["kappa"], dims)
    t_apply = time.perf_counter() - t0
    iters = max(1, min(200, int(budget_s / max(2 * t_apply, 1e-6)) - 2))
    t0 = time.perf_counter()
    _, info = oracle.cgnr(U, b1, w["kappa"], dims, tol=1e-10, max_iter=iters)
    t = time.perf_counter() - t0
    n_apply = 2 * info["iters"] + 5  # setup 2, per iteration 2, recomputed residuals 3
    gflops = n_apply * FLOP_PER_SITE * V / t / 1e9
    out = {"value": round(gflops, 4), "unit": "GFLOP/s", "cores": threads, "kind": "oracle",
           "sample": f"oracle CGNR on the same {'x'.join(map(str, dims))} lattice and source, "
                     f"{info['iters']} iterations ({n_apply} operator applications) in {t:.1f} s, "
                     f"{threads} OpenMP threads; 1320 flop/site per application",
           "dslash_gflops_all_cores": round(FLOP_PER_SITE * V / t_apply / 1e9, 4)}
    if one_core:
        # the operator on one core, at the first min(V, 65536) sites
        sites = np.arange(min(V, 65536), dtype=np.int64)
        t0 = time.perf_counter()
        oracle.apply_D_sites(U, b1, w["kappa"], dims, sites)
        t1 = time.perf_counter() - t0
        out["dslash_gflops_one_core"] = round(FLOP_PER_SITE * len(sites) / t1 / 1e9, 4)
    return out


def run_reference(args, w, rank, world):
    """The reference arm: the CPU oracle, timed per step on a bounded sample."""
    if rank != 0:
        return
    U, b = make_inputs(w, 0)
    for _ in range(args.warmup):
        cpu_baseline(w, U, b, budget_s=2.0, one_core=False)
    vals = []
    t0 = time.perf_counter()
    last = None
    for k in range(args.steps):
        last = cpu_baseline(w, U, b, budget_s=max(2.0, 60.0 / max(args.steps, 1)), one_core=k == args.steps - 1)
        vals.append(last["value"])
    el = time.perf_counter() - t0
    v = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * el / max(args.steps, 1), 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(args, w),
            "cpu_baseline": dict(last, value=round(v, 4)),
            "e2e": {"value": round(v, 4), "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


METRIC = "Dslash GFLOP/s & HBM GB/s (% roofline); CG time-to-1e-10, mixed/multi-RHS vs FP64"


def config_of(args, w):
    return {"workload": f"{args.workload}: {'x'.join(map(str, w['dims']))} {w['links']} links, kappa={w['kappa']}, "
                        f"{'12 point sources' if w['nrhs'] == 12 else 'Gaussian source'}, CGNR to true residual "
                        f"1e-10, inner precision {args.inner or w['inner']}, recon {args.recon}"
                        + (f" (inner-precision links recon {args.recon_inner})" if getattr(args, "recon_inner", None) else ""),
            "lattice": list(w["dims"]), "nrhs": w["nrhs"], "kappa": w["kappa"], "tol": 1e-10,
            "inner_prec": args.inner or w["inner"], "recon": args.recon,
            "recon_inner": getattr(args, "recon_inner", None) or args.recon,
            "preconditioner": "even-odd" if getattr(args, "eo", False) else "none",
            "l2": "flushed (512 MB write) before every timed step and every timed Dslash launch",
            "parallelism": "replicas (one independent lattice per GPU)"}


def operator_applications(r, inner: str, eo: bool) -> int:
    """Full-lattice operator applications (1320 flop/site each) of one solve from a zero
    start vector: D^dag b in the setup, 2 per iteration, 2 per FP64 reliable update and
    the two of the final FP64 check (the D x0 pair is skipped).  A mixed-precision CGNR
    solve that stopped at a reliable update uses that update as its final check.  An
    even-odd iteration applies the Schur operator twice: 4 half-lattice hops, counted as
    2 full-lattice applications."""
    n = 2 * r["iters"] + 1 + 2 * r["reliable_updates"]
    if inner == "f64" or eo:
        n += 2
    return n


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="wd", choices=["wd", "reference"])
    ap.add_argument("--workload", default="c3", choices=sorted(WORKLOADS) + ["c5"])
    ap.add_argument("--inner", default=None, choices=["f64", "f32", "f16", "df32"])
    ap.add_argument("--recon", type=int, default=18, choices=[18, 12, 8])
    ap.add_argument("--recon-inner", type=int, default=None, choices=[18, 12, 8],
                    help="link compression of the inner precision's copy (default: --recon)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--headline-only", action="store_true",
                    help="time the step and its Dslash only (no solver variants, multi-RHS block, e2e or CPU "
                         "baseline): the profiling pass")
    ap.add_argument("--delta", type=float, default=0.0, help="reliable-update threshold (0: library default)")
    ap.add_argument("--eo", action="store_true", help="even-odd preconditioned solve")
    ap.add_argument("--sweep", action="store_true",
                    help="also time the autotuned Dslash of every precision at 8^4, 12^4, 16^4, 24^4")
    ap.add_argument("--dslash-only", default=None, metavar="LX,LY,LZ,LT",
                    help="time only the Dslash kernel on this lattice (profiling helper)")
    ap.add_argument("--prec", default="f64", choices=["f64", "f32", "f16", "df32"])
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--autotune", action="store_true", help="with --dslash-only: autotune the launch shape first")
    ap.add_argument("--prefetch", action="store_true",
                    help="with --dslash-only: the FP32 kernel that prefetches neighbour spinors by cp.async")
    ap.add_argument("--tiles", default=None, metavar="ST,RT[,K]",
                    help="with --dslash-only: fix the launch shape (site tile, RHS tile, RHS per thread)")
    ap.add_argument("--staged", default=None, metavar="R,S[;R,S...]",
                    help="with --dslash-only: time the kernel with neighbour spinors staged through shared memory, "
                         "R rows per tile and S stages, for each listed pair (0: the direct-load kernel)")
    ap.add_argument("--block", action="store_true",
                    help="with --compare on c1-c3: also block CG on 12 Gaussian sources against 12 sequential solves")
    ap.add_argument("--compare", action="store_true",
                    help="c3: FP64 vs FP32 vs FP16-storage solves; c4: 12 sequential FP64 solves vs multi-RHS "
                         "and block CG; c5: batched persistent solve vs one-at-a-time FP64 solves")
    args = ap.parse_args()
    if args.workload == "c5" or (args.compare and args.impl == "wd"):
        return compare(args)
    w = WORKLOADS[args.workload]
    if args.dslash_only:
        return dslash_only(args)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo" if args.impl == "reference" else "nccl")

    if args.impl == "reference":
        run_reference(args, w, rank, world)
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    import torch
    torch.cuda.set_device(local)
    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if dist:
        dist.barrier()
    from paper_1810_04201_gb300 import wd

    inner = args.inner or w["inner"]
    nrhs = w["nrhs"]
    U, b = make_inputs(w, rank)
    lat = wd.Lattice(w["dims"])
    lat.set_gauge(U, recon=args.recon)
    if args.recon_inner and inner != "f64":
        lat.set_link_compression(wd.PRECS[inner], args.recon_inner)
    # the autotuner picks the thread-block shape of the Dslash for this lattice
    tuned = {p: lat.autotune(wd.PRECS[p], nrhs) for p in sorted({"f64", inner})}
    # and the solver autotuner the launch shape of the fused CG kernels, as the solver runs them
    tuned_cg = {p: lat.autotune_cg(wd.PRECS[p], nrhs) for p in sorted({"f64", inner})}
    fb = lat.pack(b)
    fx = lat.new_field(nrhs=nrhs)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    V = lat.V
    stream = torch.cuda.current_stream()

    def solve():
        fx.zero_()
        res, st = lat.cg(w["kappa"], fb, fx, tol=1e-10, inner=wd.PRECS[inner], nrhs=nrhs, raise_on_fail=False,
                         delta=args.delta, precondition=1 if args.eo else 0)
        return res, st

    for _ in range(args.warmup):
        solve()
    torch.cuda.synchronize()

    clocks = clock_sampler(local)
    clocks.start()
    times, launches, results = [], 0, None
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        results, st = solve()
        e1.record(stream)
        launches += lat.launches
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        if st != 0:
            raise RuntimeError(f"solve failed: {results}")
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    total_ms = float(sum(times))
    iters = max(r["iters"] for r in results)
    n_apply = max(operator_applications(r, inner, args.eo) for r in results)
    flops_step = n_apply * FLOP_PER_SITE * V * nrhs

    # ---- the Dslash kernel alone (same lattice, solve precision), CUDA events per launch
    prec = inner if inner != "f64" or nrhs == 1 else "f64"
    pid = PREC_ID[prec]
    fin = lat.pack(b, pid)
    fout = lat.new_field(pid, nrhs)
    for _ in range(3):
        lat.apply(w["kappa"], fin, fout, pid, nrhs)
    dts = []
    for _ in range(max(args.steps, 10)):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lat.apply(w["kappa"], fin, fout, pid, nrhs)
        e1.record(stream)
        torch.cuda.synchronize()
        dts.append(e0.elapsed_time(e1))
        launches += 1
    # the FP64 roof, measured in the same run and under the same clock record
    fp64_rate = wd.measure_fp64_rate()
    launches += 6
    clk = clocks.stop()
    d_ms = statistics.mean(dts)
    d_gflops = FLOP_PER_SITE * V * nrhs / (d_ms * 1e-3) / 1e9
    rprec = args.recon_inner if (args.recon_inner and prec != "f64") else args.recon
    link_b = LINK_BYTES[(prec, rprec)]
    d_bytes = V * (nrhs * 2 * SPINOR_BYTES[prec] + link_b)
    d_gbs = d_bytes / (d_ms * 1e-3) / 1e9
    peaks = load_peaks()

    # ---- end to end: canonical host buffers, copies inside the timed region
    e2e = None
    if nrhs == 1 and not args.headline_only:
        bt = torch.from_numpy(np.ascontiguousarray(b)).pin_memory()
        xt = torch.zeros_like(bt).pin_memory()
        pc = 1 if args.eo else 0
        lat.cg_canonical(w["kappa"], bt, xt, tol=1e-10, inner=wd.PRECS[inner], delta=args.delta, precondition=pc)
        et = []
        e2e_steps = max(1, min(args.steps, 3))
        for _ in range(e2e_steps):
            flush.zero_()
            xt.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            res, st = lat.cg_canonical(w["kappa"], bt, xt, tol=1e-10, inner=wd.PRECS[inner], raise_on_fail=False,
                                       delta=args.delta, precondition=pc)
            et.append(time.perf_counter() - t0)
            launches_e2e = lat.launches
        e2e_s = float(np.mean(et))
        e2e = {"value": round(flops_step / e2e_s / 1e9, 3), "unit": "GFLOP/s",
               "h2d_bytes_per_step": int(2 * bt.numel() * 16), "d2h_bytes_per_step": int(xt.numel() * 16),
               "ms_per_step": round(e2e_s * 1e3, 3), "steps": e2e_steps, "gpu_launches_per_step": int(launches_e2e),
               "call": "wd_cg_solve_canonical on pinned host buffers (b and the zero start vector in, x out)"}

    # max over ranks
    step_ms = max_over_ranks(total_ms / args.steps, dist, "cuda")
    value = job_throughput(flops_step, step_ms, world)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    if prec == "f64":
        roof = {"bound": "alu", "achieved": round(d_gflops / 1e3, 4), "peak": round(fp64_rate / 1e3, 4),
                "unit": "TFLOP/s", "frac": round(d_gflops / fp64_rate, 4),
                "peak_source": "measured in this run: FP64 multiply-add chains on every SM (wd_measure_fp64_rate)",
                "nominal_peak": round(FP64_NOMINAL_GFLOPS / 1e3, 4),
                "frac_of_nominal": round(d_gflops / FP64_NOMINAL_GFLOPS, 4),
                "hbm_achieved_gbs": round(d_gbs, 1), "hbm_frac": round(d_gbs / peaks["hbm_gbs"], 4),
                "hbm_peak_gbs": peaks["hbm_gbs"], "hbm_peak_source": peaks["source"]}
    else:
        roof = {"bound": "hbm", "achieved": round(d_gbs, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(d_gbs / peaks["hbm_gbs"], 4), "peak_source": peaks["source"]}
    kkey = f"dslash_{prec}_r{rprec}_{'x'.join(map(str, w['dims']))}_nrhs{nrhs}"
    roof["traffic"] = recorded_traffic(kkey)
    roof["kernel"] = f"wd::dslash_kernel<{pid},{rprec},false,EpXpay> ({kkey})"
    roof["algorithmic_bytes_per_launch"] = d_bytes
    roof["algorithmic_flops_per_launch"] = FLOP_PER_SITE * V * nrhs
    roof["avg_launch_ms"] = round(d_ms, 5)
    roof["dslash_gflops"] = round(d_gflops, 2)
    roof["dslash_hbm_gbs"] = round(d_gbs, 1)

    line = {"metric": METRIC, "value": round(value, 3), "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(step_ms, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if inner == "f64" else f"{inner}+f64", "data": "synthetic",
            "config": config_of(args, w),
            "cg": {"time_to_solution_ms": round(step_ms, 4), "iterations": iters,
                   "reliable_updates": max(r["reliable_updates"] for r in results),
                   "true_rel_resid": max(r["true_rel_resid"] for r in results),
                   "true_rel_resid_b": max(r["true_rel_resid_b"] for r in results),
                   "operator_applications": n_apply},
            "roofline": roof, "clocks": clk, "gpu_launches": int(launches),
            "autotuned_tiles": {p: {"site_tile": t[0], "rhs_tile": t[1]} for p, t in tuned.items()},
            "autotuned_cg_tiles": {p: {"site_tile": t[0], "rhs_tile": t[1]} for p, t in tuned_cg.items()},
            "e2e": e2e}
    if not args.headline_only and nrhs == 1 and world == 1:
        line["cg"]["variants"] = cg_variants(wd, torch, lat, w, fb, fx, flush, step_ms, args)
        if args.workload == "c3":
            lat.close()
            line["multi_rhs"] = multi_rhs_block(wd, torch, flush, args)
    if args.sweep:
        line["dslash_sweep"] = sweep(wd, torch, flush, stream, args.recon)
    if not args.no_cpu_baseline and not args.headline_only and rank == 0:
        line["cpu_baseline"] = cpu_baseline(w, U, b)
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def _median_solve_ms(torch, flush, fn, reps):
    """Median device time (CUDA events) of fn over reps runs after one warm-up, L2 flushed
    before each; returns (ms, last result)."""
    out = fn()
    ts = []
    for _ in range(reps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts), out


# (name, inner precision, even-odd, inner-precision link compression, stop rule)
CG_VARIANTS = (("f32", "f32", 0, None, 0), ("f16", "f16", 0, None, 0), ("df32", "df32", 0, None, 0),
               ("f64_eo", "f64", 1, None, 0), ("f32_eo", "f32", 1, None, 0), ("f16_eo", "f16", 1, None, 0),
               ("df32_eo", "df32", 1, None, 0), ("f32_recon12_inner", "f32", 0, 12, 0),
               ("f32_eo_recon12_inner", "f32", 1, 12, 0), ("f16_eo_recon12_inner", "f16", 1, 12, 0),
               ("f64_system_rule", "f64", 0, None, 1), ("f32_eo_recon12_inner_system_rule", "f32", 1, 12, 1))


def cg_variants(wd, torch, lat, w, fb, fx_f64, flush, f64_ms, args):
    """Every solver variant on the step's lattice and source: time to a true FP64 residual of
    1e-10 (normal residual; the system rule: |b - D x| / |b|), against the FP64 step."""
    x64 = lat.unpack(fx_f64)
    for p in sorted({v[1] for v in CG_VARIANTS} - {"f64"}):
        lat.autotune_cg(wd.PRECS[p], 1)
    reps = 3
    out = {"reps": f"median of {reps} after one warm-up, L2 flushed before each",
           "reference": f"plain FP64 CGNR step, {round(f64_ms, 3)} ms"}
    for name, inner, eo, rin, rule in CG_VARIANTS:
        pid = wd.PRECS[inner]
        if rin:
            lat.set_link_compression(pid, rin)
        fx = lat.new_field()

        def solve():
            fx.zero_()
            return lat.cg(w["kappa"], fb, fx, tol=1e-10, inner=pid, raise_on_fail=False, precondition=eo,
                          stop_rule=rule)

        ms, (res, st) = _median_solve_ms(torch, flush, solve, reps)
        r = res[0]
        out[name] = {"ms": round(ms, 3), "speedup_vs_f64": round(f64_ms / ms, 3), "iters": r["iters"],
                     "reliable_updates": r["reliable_updates"], "inner_corrections": r["inner_corrections"],
                     "status": st,
                     "true_rel_resid": r["true_rel_resid"], "true_rel_resid_b": r["true_rel_resid_b"],
                     "rel_diff_vs_f64_solution": rel_diff(lat.unpack(fx), x64)}
        if rin:
            lat.set_link_compression(pid, args.recon)
        del fx
    return out


def multi_rhs_block(wd, torch, flush, args):
    """The 12 spin-colour point sources of the 24^3 x 48 workload: one multi-RHS solve against
    12 sequential FP64 solves, each to a true FP64 residual of 1e-10."""
    w = WORKLOADS["c4"]
    U, B = make_inputs(w, 0)
    lat = wd.Lattice(w["dims"])
    lat.set_gauge(U, recon=args.recon)
    for p in ("f64", "f32"):
        for n in (1, 12):
            lat.autotune(wd.PRECS[p], n)
            lat.autotune_cg(wd.PRECS[p], n)
    fb = lat.pack(B)
    fbs = [lat.pack(B[k]) for k in range(12)]
    fys = [lat.new_field() for _ in range(12)]
    reps = 2

    def seq():
        res = []
        for k in range(12):
            fys[k].zero_()
            res.append(lat.cg(w["kappa"], fbs[k], fys[k], tol=1e-10)[0][0])
        return res

    ms_seq, res_seq = _median_solve_ms(torch, flush, seq, reps)
    Xs = [lat.unpack(f) for f in fys]
    out = {"workload": "c4: 24x24x24x48 haar links, kappa=0.12, 12 point sources at the origin",
           "reps": f"median of {reps} after one warm-up",
           "sequential_f64": {"ms": round(ms_seq, 3), "iters_max": max(r["iters"] for r in res_seq),
                              "max_true_rel_resid": max(r["true_rel_resid"] for r in res_seq)}}
    for name, inner, eo, rin in (("multi_rhs_f64", "f64", 0, None), ("multi_rhs_f32", "f32", 0, None),
                                 ("multi_rhs_f32_eo_recon12_inner", "f32", 1, 12)):
        pid = wd.PRECS[inner]
        if rin:
            lat.set_link_compression(pid, rin)
        fx = lat.new_field(nrhs=12)

        def solve():
            fx.zero_()
            return lat.cg(w["kappa"], fb, fx, tol=1e-10, inner=pid, nrhs=12, raise_on_fail=False, precondition=eo)

        ms, (res, st) = _median_solve_ms(torch, flush, solve, reps)
        X = lat.unpack(fx, nrhs=12, squeeze=False)
        out[name] = {"ms": round(ms, 3), "speedup_vs_sequential_f64": round(ms_seq / ms, 3), "status": st,
                     "iters_max": max(r["iters"] for r in res),
                     "max_true_rel_resid": max(r["true_rel_resid"] for r in res),
                     "max_rel_diff_vs_sequential": max(rel_diff(X[k], Xs[k]) for k in range(12))}
        if rin:
            lat.set_link_compression(pid, args.recon)
        del fx
    lat.close()
    return out


def rel_diff(a, b) -> float:
    """||a - b|| / ||b|| of two solutions."""
    nb = np.linalg.norm(np.ravel(b))
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / (nb if nb > 0 else 1.0))


def _timed_solves(torch, fn, reps):
    """Median device time (CUDA events) of `fn` over `reps` runs after one warm-up."""
    fn()
    ts = []
    out = None
    for _ in range(reps):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return statistics.median(ts), out


def compare(args):
    """Solver comparisons on one GPU (one JSON line with a `compare` object)."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1810_04201_gb300 import gen, wd
    reps = max(1, min(args.steps, 3))
    line = {"workload": args.workload, "compare": {}}
    if args.workload == "c5":
        shapes, kappas, seeds = gen.batch_workload(64)
        lats, bs, xs = [], [], []
        for dims, seed in zip(shapes, seeds):
            lat = wd.Lattice(dims)
            lat.set_gauge(gen.haar_links(dims, seed), recon=args.recon)
            if args.recon_inner:
                lat.set_link_compression(wd.WD_F32, args.recon_inner)
            lats.append(lat)
            bs.append(lat.pack(gen.gaussian_source(dims, seed)))
            xs.append(lat.new_field())
        V = sum(l.V for l in lats)

        def batched():
            for x in xs:
                x.zero_()
            return wd.cg_batched(lats, kappas, bs, xs, tol=1e-10, inner=wd.WD_F32)

        ms_b, (res_b, st_b) = _timed_solves(torch, batched, reps)
        xb = [l.unpack(x) for l, x in zip(lats, xs)]
        ys = [l.new_field() for l in lats]

        def one_by_one():
            out = []
            for l, k, b, y in zip(lats, kappas, bs, ys):
                y.zero_()
                out.append(l.cg(k, b, y, tol=1e-10)[0][0])
            return out

        ms_s, res_s = _timed_solves(torch, one_by_one, reps)
        err = max(rel_diff(a, l.unpack(y)) for a, l, y in zip(xb, lats, ys))
        line["compare"] = {
            "lattices": 64, "total_sites": V, "recon": args.recon, "recon_inner": args.recon_inner or args.recon,
            "shapes": sorted(set("x".join(map(str, d)) for d in shapes)),
            "batched_mixed_f32": {"ms": round(ms_b, 3), "solves_per_s": round(64e3 / ms_b, 1),
                                  "per_solve_latency_ms": round(ms_b, 3), "status": st_b,
                                  "max_true_rel_resid": max(r["true_rel_resid"] for r in res_b),
                                  "iters_min_max": [min(r["iters"] for r in res_b), max(r["iters"] for r in res_b)],
                                  "gpu_launches": 1},
            "one_at_a_time_f64": {"ms": round(ms_s, 3), "solves_per_s": round(64e3 / ms_s, 1),
                                  "per_solve_latency_ms": round(ms_s / 64, 3),
                                  "max_true_rel_resid": max(r["true_rel_resid"] for r in res_s)},
            "speedup_batched_vs_f64": round(ms_s / ms_b, 3),
            "max_rel_diff_batched_vs_f64_solutions": err,
            "note": "per-solve latency of the batched launch = time until all 64 solutions are ready"}
        print(json.dumps(line))
        return
    w = WORKLOADS[args.workload]
    U, b = make_inputs(w, 0)
    dims = w["dims"]
    lat = wd.Lattice(dims)
    lat.set_gauge(U, recon=args.recon)
    if args.recon_inner:
        for p in (wd.WD_F32, wd.WD_F16, wd.WD_DF32):
            lat.set_link_compression(p, args.recon_inner)
    V = lat.V
    if args.workload in ("c1", "c2", "c3"):
        fb = lat.pack(b)
        variants = {"f64": (wd.WD_F64, 0), "f32": (wd.WD_F32, 0), "f16": (wd.WD_F16, 0), "df32": (wd.WD_DF32, 0),
                    "f64_eo": (wd.WD_F64, 1), "f32_eo": (wd.WD_F32, 1), "f16_eo": (wd.WD_F16, 1),
                    "df32_eo": (wd.WD_DF32, 1)}
        sols = {}
        for name, (inner, eo) in variants.items():
            fx = lat.new_field()

            def solve():
                fx.zero_()
                return lat.cg(w["kappa"], fb, fx, tol=1e-10, inner=inner, raise_on_fail=False, precondition=eo)

            ms, (res, st) = _timed_solves(torch, solve, reps)
            r = res[0]
            x = lat.unpack(fx)
            sols[name] = x
            line["compare"][name] = {"ms": round(ms, 3), "iters": r["iters"], "reliable_updates": r["reliable_updates"],
                                     "inner_corrections": r["inner_corrections"],
                                     "status": st, "true_rel_resid_normal": r["true_rel_resid"],
                                     "true_rel_resid_b": r["true_rel_resid_b"],
                                     "gflops": round((2 * r["iters"] + 4 + 2 * r["reliable_updates"]
                                                      + 2 * r["inner_corrections"]) * 1320 * V
                                                     / ms / 1e6, 1)}
        for name in variants:
            if name == "f64":
                continue
            line["compare"][name]["rel_diff_vs_f64_solution"] = rel_diff(sols[name], sols["f64"])
            line["compare"][name]["speedup_vs_f64"] = round(line["compare"]["f64"]["ms"] / line["compare"][name]["ms"], 3)
        if args.block:
            line["compare"]["block_cg_12_sources"] = block_vs_sequential(wd, torch, lat, w, reps)
        line["note"] = ("gflops counts 1320 flop/site per full-lattice operator application; an even-odd "
                        "iteration applies the Schur operator twice, counted as 2 * 1320 * V / 2 * 2 flop")
    else:  # c4: 12 point sources
        B = b
        fb = lat.pack(B)
        fbs = [lat.pack(B[k]) for k in range(12)]
        fys = [lat.new_field() for _ in range(12)]

        def seq():
            res = []
            for k in range(12):
                fys[k].zero_()
                res.append(lat.cg(w["kappa"], fbs[k], fys[k], tol=1e-10)[0][0])
            return res

        ms, res = _timed_solves(torch, seq, reps)
        Xs = np.stack([lat.unpack(f) for f in fys])
        line["compare"]["sequential_f64"] = {"ms": round(ms, 3), "iters_max": max(r["iters"] for r in res),
                                            "max_true_rel_resid": max(r["true_rel_resid"] for r in res)}
        for name, inner, block, eo in (("multi_rhs_f64", wd.WD_F64, 0, 0), ("multi_rhs_f32", wd.WD_F32, 0, 0),
                                       ("multi_rhs_f16", wd.WD_F16, 0, 0), ("multi_rhs_df32", wd.WD_DF32, 0, 0),
                                       ("multi_rhs_f32_eo", wd.WD_F32, 0, 1), ("multi_rhs_f64_eo", wd.WD_F64, 0, 1),
                                       ("block_cg_f64", wd.WD_F64, 1, 0)):
            fx = lat.new_field(nrhs=12)

            def solve():
                fx.zero_()
                return lat.cg(w["kappa"], fb, fx, tol=1e-10, inner=inner, nrhs=12, block=block, raise_on_fail=False,
                              precondition=eo)

            ms2, (res2, st2) = _timed_solves(torch, solve, reps)
            X = lat.unpack(fx, nrhs=12, squeeze=False)
            line["compare"][name] = {"ms": round(ms2, 3), "status": st2, "iters_max": max(r["iters"] for r in res2),
                                     "max_true_rel_resid": max(r["true_rel_resid"] for r in res2),
                                     "speedup_vs_sequential_f64": round(ms / ms2, 3),
                                     "max_rel_diff_vs_sequential": max(rel_diff(X[k], Xs[k]) for k in range(12))}
    line["config"] = config_of(args, w)
    print(json.dumps(line))


def block_vs_sequential(wd, torch, lat, w, reps):
    """Block CG (one Krylov space for 12 Gaussian sources, FP64) against 12 sequential FP64
    solves on the same lattice, each to a true normal residual of 1e-10."""
    from paper_1810_04201_gb300 import gen
    B = np.stack([gen.gaussian_source(w["dims"], w["seed"] + 100 + k) for k in range(12)])
    fb = lat.pack(B)
    fbs = [lat.pack(B[k]) for k in range(12)]
    fys = [lat.new_field() for _ in range(12)]

    def seq():
        out = []
        for k in range(12):
            fys[k].zero_()
            out.append(lat.cg(w["kappa"], fbs[k], fys[k], tol=1e-10)[0][0])
        return out

    ms_seq, res_seq = _timed_solves(torch, seq, reps)
    fx = lat.new_field(nrhs=12)

    def blk():
        fx.zero_()
        return lat.cg(w["kappa"], fb, fx, tol=1e-10, nrhs=12, block=1, raise_on_fail=False)

    ms_blk, (res_blk, st) = _timed_solves(torch, blk, reps)
    X = lat.unpack(fx, nrhs=12, squeeze=False)
    return {"sequential_f64_ms": round(ms_seq, 3), "sequential_iters_max": max(r["iters"] for r in res_seq),
            "block_cg_f64_ms": round(ms_blk, 3), "block_iters": max(r["iters"] for r in res_blk), "status": st,
            "block_max_true_rel_resid": max(r["true_rel_resid"] for r in res_blk),
            "speedup_block_vs_sequential": round(ms_seq / ms_blk, 3),
            "max_rel_diff_vs_sequential": max(rel_diff(X[k], lat.unpack(fys[k])) for k in range(12))}


def dslash_only(args):
    """W warm-up and K timed launches of one Dslash (D, xpay) on a Haar lattice; with
    --staged "R,S;R,S;..." each listed configuration of the staged kernel (R rows per tile,
    S stages; "0" the direct-load kernel) is timed in turn, one JSON line each."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1810_04201_gb300 import gen, wd
    dims = tuple(int(x) for x in args.dslash_only.split(","))
    lat = wd.Lattice(dims)
    lat.set_gauge(gen.haar_links(dims, 3), recon=args.recon)
    b = gen.gaussian_source(dims, 4, nrhs=args.nrhs)
    pid = PREC_ID[args.prec]
    tuned = lat.autotune(pid, args.nrhs) if args.autotune else None
    if args.tiles:
        t = [int(v) for v in args.tiles.split(",")]
        lat.set_tiles(pid, args.nrhs, t[0], t[1])
        if len(t) > 2:
            lat.set_rhs_per_thread(pid, args.nrhs, t[2])
        tuned = list(lat.tiles(pid, args.nrhs))
    if args.prefetch:
        lat.set_prefetch(pid, True)
        tuned = {"tiles": list(lat.tiles(pid, args.nrhs)), "prefetch": True}
    fi = lat.pack(b if args.nrhs > 1 else b[0], pid)
    fo = lat.new_field(pid, args.nrhs)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    configs = [[int(v) for v in c.split(",")] for c in args.staged.split(";")] if args.staged else [[0]]
    for cfg in configs:
        rows, stages = cfg[0], (cfg[1] if len(cfg) > 1 else 2)
        lat.set_staging(pid, rows, stages) if rows else lat.set_staging(pid, 0)
        tiles = {"staged_rows": rows, "stages": stages} if rows else tuned
        for _ in range(args.warmup):
            lat.apply(0.12, fi, fo, pid, args.nrhs)
        ts = []
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lat.apply(0.12, fi, fo, pid, args.nrhs)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = statistics.mean(ts)
        if rows and lat.staging_error():
            raise RuntimeError("a wait of the staged kernel ran out")
        V = lat.V
        nb = V * (args.nrhs * 2 * SPINOR_BYTES[args.prec] + LINK_BYTES[(args.prec, args.recon)])
        print(json.dumps({"dslash": list(dims), "prec": args.prec, "recon": args.recon, "nrhs": args.nrhs,
                          "tiles": tiles, "ms": round(ms, 5), "gflops": round(FLOP_PER_SITE * V * args.nrhs / ms / 1e6, 1),
                          "algorithmic_gbs": round(nb / ms / 1e6, 1), "bytes_per_launch": nb}), flush=True)


def sweep(wd, torch, flush, stream, recon):
    from paper_1810_04201_gb300 import gen
    out = {}
    for L in (8, 12, 16, 24):
        dims = (L, L, L, L)
        lat = wd.Lattice(dims)
        lat.set_gauge(gen.haar_links(dims, 3), recon=recon)
        b = gen.gaussian_source(dims, 4)
        row = {}
        for prec, pid in (("f64", 0), ("f32", 1), ("f16", 2), ("df32", 3)):
            tiles = lat.autotune(pid, 1)
            fi = lat.pack(b, pid)
            fo = lat.new_field(pid)
            for _ in range(3):
                lat.apply(0.12, fi, fo, pid)
            ts = []
            for _ in range(10):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                lat.apply(0.12, fi, fo, pid)
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            ms = statistics.mean(ts)
            V = lat.V
            row[prec] = {"ms": round(ms, 5), "gflops": round(FLOP_PER_SITE * V / ms / 1e6, 1),
                         "gbs": round(V * dslash_bytes(prec, recon) / ms / 1e6, 1),
                         "site_tile": tiles[0]}
        out[f"{L}^4"] = row
        lat.close()
    return out


if __name__ == "__main__":
    main()
