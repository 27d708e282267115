"""Benchmark: SDP solves/s and p50/p99 latency at 1e-6 relative duality gap, the
mixed-precision form against the plain FP64 PCG method on the same GB300.

Default workload ("batched"): the first 16 instances of the batched
matrix-completion workload (p, q uniform in [50, 400], r uniform in {1..4},
m = min(pq/2, ceil(3 r (p+q) ln(p+q))) uniform observations, seeds 4000..4015).
One step solves all 16 SDPs, each from the interior-point start point to
relative gap, primal and dual infeasibility <= 1e-6 with every Newton system
solved to a 1e-8 FP64 true relative residual.  The problems are advanced in
lockstep (sdp_batch_solve): their dense phases on one stream and host thread
each, every PCG iteration of all their Newton systems as one sequence of batched
launches under a CUDA graph.  The problem data stay in HBM across steps; each
solve resets its iterate on the device; a 256 MB write flushes L2 between steps.

Two arms run on the same instances (--arms, default "fp32,fp64"): the mixed form
(FP32 split matvec and FP32 core inverse inside PCG, FP64 refinement and FP64
everything else) and the plain FP64 form.  The first arm is the headline `value`;
`arms` carries both, each with solves/s, per-problem p50/p99 latency (start of
the batched solve to the end of the problem's last iteration), iteration counts
and its error against the FP64 arm and the planted matrix.

Other workloads: C2 (n = 1000, m = 8000, rank 2; --k-max/--eta for the adaptive
split rank), C3 (n = 4000, m = 60,000, rank 3), fig2 (p = q = 500, rank 4,
m = 20,000: the paper's Fig. 2 instance), serving (the request stream).

The printed line (rank 0) carries the contract keys plus: roofline (the batched
FP64 matvec, timed with CUDA events in an instrumented host-driven step after the
timed ones) and rooflines of the other kernel classes, cpu_baseline (measured
full oracle solves of the workload's smallest instances on the host cores), e2e
(host triplets -> sdp_setup -> solve -> solution copied back, through the public
API, headline arm), clocks (nvidia-smi samples taken during the timed region) and
gpu_launches (library kernels launched in the timed region).

--impl reference times the FP64 oracle (explicit Hessian + Cholesky) on the host
cores.  Under torchrun (--gpus N) each rank solves its own 16 instances (ranks
take distinct blocks of the 256) with no collective on the data path; the step
time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import queue
import statistics
import subprocess
import tempfile
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "SDP solves/s + p50/p99 latency at 1e-6 gap: served/mixed vs plain FP64 PCG"
UNIT = "solves/s"
DTYPES = {"fp64": "f64", "fp32": "f32+f64 (mixed)", "bf16": "bf16+f32+f64 (mixed)"}
FORMS = {"fp64": "plain FP64 PCG",
         "fp32": "mixed: FP32 split matvec + FP32 core inverse in PCG, FP64 refinement and IPM",
         "bf16": "mixed: BF16 split W_s (FP32 accumulation) + FP32 core inverse in PCG, FP64 refinement and IPM"}

# FP32 FMA peak derived the same way: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP32_PEAK_SOURCE = "derived: 152 SMs x 128 FP32 FMA/clk x 2 flop x 2.07 GHz"
FP32_CLASSES = ("matvec_lp_b",)

# FP64 FMA throughput of this GB300, measured with a register-resident DFMA
# loop (1216 CTAs x 256 threads, 8 independent chains per thread): 1.194 TFLOP/s.
# Nominal from the unit count: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz = 1.26.
# FP64 peak of the GB300 derived from unit counts and clock: 152 SMs x 2 FP64 FMA
# per clock per SM x 2 flop x 2.07 GHz (an FMA-chain probe reached 95% of it)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP64_PEAK_SOURCE = "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz"

ALU_CLASSES = ("matvec_b", "gemm_f64", "sytrd", "potrf", "trsm")
PHASES = ("nt_scaling", "precond_build", "pcg", "max_step", "lanczos")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def _dist():
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


class Clocks:
    """nvidia-smi samples (200 ms) during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.environ.get("SDP_CLOCKS_CSV") or os.path.join(tempfile.gettempdir(),
                                                                     f"sdp_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                p = [x.strip() for x in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    mx.append(float(p[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, p[5:9]):
                    if v.lower() in ("active", "1"):
                        reasons.add(nm)
        except Exception:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def shard_indices(rank, world, count, total=256):
    """Instances of the batched set solved by `rank`: a contiguous block of `count`,
    distinct across ranks (weak scaling: every rank solves its own `count` SDPs)."""
    start = (rank * count) % total
    return [(start + i) % total for i in range(count)]


def max_over_ranks(value, dist, device):
    """The largest `value` over all ranks (the whole job ends with the slowest rank)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload(name, count, rank=0, world=1):
    import sdp_inputs as si
    if name == "C2":
        d = si.config_instance("C2")
        return [d], "matrix-completion SDP n1=n2=500 (n=1000), rank 2, m=8000, seed 2"
    if name == "C3":
        d = si.config_instance("C3")
        return [d], "matrix-completion SDP n1=n2=2000 (n=4000), rank 3, m=60000, seed 3"
    if name == "fig2":
        d = si.mc_instance(500, 500, 4, 20000, 1702)
        return [d], ("matrix-completion SDP p=q=500 (n=1000), rank 4, m=20000, seed 1702 "
                     "(the instance shape of the paper's Fig. 2)")
    all_specs = si.batched_specs(256)
    idx = shard_indices(rank, world, count)
    specs = [all_specs[i] for i in idx]
    inst = [si.mc_instance(s["p"], s["q"], s["r"], s["m"], s["seed"]) for s in specs]
    first = specs[0]["seed"]
    desc = (f"batched matrix completion: {count} of the 256 batched instances per rank "
            f"(p,q~U[50,400], r~U{{1..4}}, m=min(pq/2, 3r(p+q)ln(p+q)), rank 0 seeds {first}..{first + count - 1}); "
            f"n {min(d.n for d in inst)}..{max(d.n for d in inst)}, m {min(d.m for d in inst)}.."
            f"{max(d.m for d in inst)}")
    return inst, desc


def oracle_sample(insts, budget_s=25.0):
    """Measured oracle baseline: full FP64 oracle solves (explicit m x m Hessian and
    Cholesky per Newton system) of the workload's smallest instances, smallest
    first, until about budget_s of host time.  Returns (solves/s over the sampled
    instances, description, per-instance records).  Nothing is extrapolated."""
    from oracle import sdp_oracle as o
    done, used = 0.0, []
    for d in sorted(insts, key=lambda d: d.m):
        P = o.Problem.from_data(d)
        t0 = time.perf_counter()
        r = o.ipm_solve(P)
        el = time.perf_counter() - t0
        done += el
        used.append(dict(n=d.n, m=d.m, seconds=el, ipm_iters=len(r.log), converged=bool(r.converged)))
        if done > budget_s:
            break
    rate = len(used) / done
    sample = (f"full oracle solves (NumPy/LAPACK FP64, explicit m x m Hessian + Cholesky) of the {len(used)} "
              f"smallest of the {len(insts)} workload instances (n {used[0]['n']}..{used[-1]['n']}, m "
              f"{used[0]['m']}..{used[-1]['m']}), {done:.1f} s in total; solves/s of that sample, not of the "
              f"whole workload (the largest instance, m = {max(d.m for d in insts)}, needs an "
              f"{8 * max(d.m for d in insts) ** 2 / 1e9:.0f} GB Hessian)")
    return rate, sample, used


def run_reference(args):
    """The oracle as the reference arm, timed on the machine's host cores: warm-up runs one
    full oracle solve of the workload's smallest instance (its IPM iteration count);
    each timed step is one oracle IPM iteration of that instance, and the value is
    1 / (mean iteration time x iteration count), solves/s of that instance."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    insts, desc = workload(args.workload, args.batch)
    from oracle import sdp_oracle as o
    small = sorted(insts, key=lambda d: d.m)[0]
    P = o.Problem.from_data(small)
    t0 = time.perf_counter()
    full = o.ipm_solve(P)
    full_s = time.perf_counter() - t0
    its = len(full.log)
    for _ in range(max(0, args.warmup - 1)):
        o.ipm_solve(P, o.IPMParams(maxit=1))
    times = []
    for _ in range(args.steps):
        t1 = time.perf_counter()
        o.ipm_solve(P, o.IPMParams(maxit=1))
        times.append(time.perf_counter() - t1)
    per_iter = statistics.mean(times)
    value = 1.0 / (per_iter * its)
    sample = (f"oracle (NumPy/LAPACK FP64, explicit Hessian + Cholesky) on the workload's smallest instance "
              f"(n={small.n}, m={small.m}): one IPM iteration per step ({per_iter:.2f} s) x {its} iterations of "
              f"its measured full solve ({full_s:.1f} s, converged={bool(full.converged)})")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * per_iter, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": desc, "instances_timed": 1, "l2_flush": False, "same_config": False,
                       "fits_in_driver_run": True, "oracle_full_solve_s": full_s, "oracle_ipm_iters": its},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": _cores(), "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _pct(xs, q):
    srt = sorted(xs)
    return srt[min(len(srt) - 1, max(0, int(math.ceil(q * len(srt))) - 1))]


def _recovered(d, X):
    """The p x q block Z of X for a matrix-completion instance (None otherwise)."""
    p = d.meta.get("p") if isinstance(d.meta, dict) else None
    return None if p is None else X[:p, p:]


class Arm:
    """One precision form of the workload: its problems resident on the device, a
    lockstep batch over them, and the timings of its steps."""

    def __init__(self, args, insts, prec, kk):
        import torch
        from paper_1703_10973_gb300 import SDPBatch, SDPProblem, default_params
        self.prec = prec
        self.args = args
        self.insts = insts
        extra = {"inner_rtol_lp": args.inner_lp} if args.inner_lp > 0 else {}
        self.params = default_params(prec=prec, k=kk, pcg_maxit=args.pcg_maxit, pcg_graph=args.pcg_graph,
                                     k_max=args.k_max, eta=args.eta, **extra)
        n = len(insts) if args.batched_launch else min(args.streams, len(insts))
        self.streams = [torch.cuda.Stream() for _ in range(n)]
        self.probs = [SDPProblem.from_data(d, params=self.params, stream=self.streams[i % n].cuda_stream)
                      for i, d in enumerate(insts)]
        self.batch = None
        self.bstream = torch.cuda.Stream(priority=-1)   # PCG stages ahead of the dense phases
        if args.batched_launch:
            self.batch = SDPBatch(self.probs, stream=self.bstream.cuda_stream, groups=args.batch_groups)
        self.step_ms, self.lat_ms, self.res = [], [], None
        self.stage_ms = {}

    def solve_once(self, start_event=None):
        """Solve every instance once from the start point; returns (per-solve ms, results)."""
        import torch
        if start_event is not None:
            self.bstream.wait_event(start_event)
            for st in self.streams:
                st.wait_event(start_event)
        if self.batch is not None:
            torch.cuda.synchronize()
            for p in self.probs:
                p.reset()
            res = self.batch.solve(allow_maxit=True)
            torch.cuda.synchronize()
            self.stage_ms = {k: (round(v * 1e3, 1) if k not in ("graph_launches", "batched_iters") else int(v))
                             for k, v in self.batch.stage_seconds().items()}
            # per problem: host wall time from the start of the batched solve to the
            # end of that problem's last interior-point iteration
            return [1e3 * r["seconds"] for r in res], res
        lat = [None] * len(self.probs)
        res = [None] * len(self.probs)
        errs = []
        nst = len(self.streams)

        def worker(s):
            try:
                st = self.streams[s]
                for i in range(s, len(self.probs), nst):
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record(st)
                    self.probs[i].reset()
                    res[i] = self.probs[i].solve(allow_maxit=True)
                    b.record(st)
                    b.synchronize()
                    lat[i] = a.elapsed_time(b)
            except Exception as e:  # surfaced after join
                errs.append(e)

        th = [threading.Thread(target=worker, args=(s,)) for s in range(nst)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        if errs:
            raise errs[0]
        return lat, res

    def timed(self, flush, steps, dist):
        import torch
        for i in range(steps):
            flush.fill_(float(i))          # evict L2 between steps (256 MB > 126 MB L2)
            torch.cuda.synchronize()
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record()
            lat, res = self.solve_once(t0)
            for s in self.streams + [self.bstream]:   # join every stream into the default stream
                torch.cuda.current_stream().wait_stream(s)
            t1.record()
            torch.cuda.synchronize()
            self.step_ms.append(t0.elapsed_time(t1))
            self.lat_ms += lat
            self.res = res

    def solutions(self):
        return [p.get_solution()[0] for p in self.probs]

    def close(self):
        if self.batch is not None:
            self.batch.close()
        for p in self.probs:
            p.close()


def instrumented_step(args, insts, prec, kk, stream):
    """One lockstep solve of the workload with CUDA events around every kernel class
    and phase.  The batched PCG runs inside a graph whose kernels events cannot
    bracket, so this step drives the same batched kernels from the host
    (pcg_graph = 0), all problems in one lockstep group (nothing runs beside the
    batched matvec)."""
    import torch
    from paper_1703_10973_gb300 import SDPBatch, SDPProblem, default_params
    ip = default_params(prec=prec, k=kk, pcg_maxit=args.pcg_maxit, pcg_graph=0, k_max=args.k_max, eta=args.eta)
    streams = [torch.cuda.Stream() for _ in insts]
    probs = [SDPProblem.from_data(d, params=ip, stream=streams[i].cuda_stream) for i, d in enumerate(insts)]
    ib = SDPBatch(probs, stream=stream.cuda_stream, groups=1)
    torch.cuda.synchronize()
    probs[0].timing_enable("*")
    t0 = time.perf_counter()
    ib.solve(allow_maxit=True)
    torch.cuda.synchronize()
    wall = (time.perf_counter() - t0) * 1e3
    rep = probs[0].timing_report()
    probs[0].timing_enable(None)
    ib.close()
    for p in probs:
        p.close()
    return rep, wall


# All-active batched FP64 matvec of the 16 bench instances: algorithmic flops
# (2 nnz(V) n + 2 nent n summed) and the DRAM bytes ncu measured for its SpMM and SDDMM.
MATVEC_B_ALL_ACTIVE_FLOPS = 0.558157e9 + 0.279079e9
MATVEC_B_NCU_BYTES = 36.78e6 + 36.97e6


def roofline_of(cls, rep, wall):
    """Roofline object of kernel class `cls` from the instrumented step's records."""
    kt = rep.get(cls)
    if not kt or not kt[1]:
        return None
    ms, cnt, fl, by = kt
    common = {"kernel": cls, "launches": cnt, "avg_us": 1e3 * ms / cnt, "busy_ms_per_step": ms,
              "step_ms_instrumented": wall, "traffic": None}
    if cls in FP32_CLASSES:
        ach = fl / (ms * 1e-3) / 1e12
        return dict(common, bound="alu", achieved=ach, peak=FP32_PEAK_TFLOPS, unit="TFLOP/s",
                    frac=ach / FP32_PEAK_TFLOPS, peak_source=FP32_PEAK_SOURCE,
                    hbm_gbs=by / (ms * 1e-3) / 1e9)
    if cls in ALU_CLASSES:
        ach = fl / (ms * 1e-3) / 1e12
        return dict(common, bound="alu", achieved=ach, peak=FP64_PEAK_TFLOPS, unit="TFLOP/s",
                    frac=ach / FP64_PEAK_TFLOPS, peak_source=FP64_PEAK_SOURCE)
    peak = _peaks().get("hbm_gbs", 6776.3)
    ach = by / (ms * 1e-3) / 1e9
    return dict(common, bound="hbm", achieved=ach, peak=peak, unit="GB/s", frac=ach / peak,
                peak_source="measured copy bandwidth (MEASURED_PEAKS.json)")


def run(args):
    import torch
    ws, rank, local = _dist()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1703_10973_gb300 import SDPProblem, _build, load
    if not os.path.exists(_build.LIB):
        _build.build()
    load()
    insts, desc = workload(args.workload, args.batch, rank, ws)
    kk = args.k
    precs = [x for x in args.arms.split(",") if x]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    arms = [Arm(args, insts, prec, kk) for prec in precs]

    for arm in arms:
        for _ in range(args.warmup):
            arm.solve_once()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    probe = arms[0].probs[0]
    launches = {}
    with Clocks(local) as clk:
        for arm in arms:
            l0 = probe.launch_count()
            arm.timed(flush, args.steps, dist)
            launches[arm.prec] = probe.launch_count() - l0
    per_arm = {}
    for arm in arms:
        total_ms = sum(arm.step_ms)
        if dist is not None:
            total_ms = max_over_ranks(total_ms, dist, "cuda")
        per_arm[arm.prec] = total_ms
    if dist is not None:
        dist.barrier()
    head = arms[0]
    solves = len(insts) * args.steps * ws
    value = solves / (per_arm[head.prec] / 1e3)

    # ---- each arm against the plain FP64 arm (same instances, same seed)
    ref_arm = next((a for a in arms if a.prec == "fp64"), None)
    ref_X = ref_arm.solutions() if ref_arm is not None else None
    arm_lines = {}
    for arm in arms:
        Xs = arm.solutions()
        res = arm.res
        line = {"value": solves / (per_arm[arm.prec] / 1e3), "unit": UNIT,
                "ms_per_step": per_arm[arm.prec] / args.steps,
                "latency_ms": {"p50": _pct(arm.lat_ms, 0.50), "p99": _pct(arm.lat_ms, 0.99),
                               "what": ("per problem: start of the batched solve -> end of its last IPM "
                                        "iteration" if arm.batch is not None else
                                        "per solve: CUDA events around the solve on its stream")},
                "converged": all(r["converged"] for r in res),
                "max_relgap": max(r["relgap"] for r in res),
                "ipm_iters_mean": float(np.mean([r["iters"] for r in res])),
                "pcg_iters_per_solve_mean": float(np.mean([r["pcg_iters_total"] for r in res])),
                "gpu_launches": int(launches[arm.prec]),
                "stage_ms_last_step": arm.stage_ms or None,
                "spmm_autotune": ({"rows_per_cta": arm.batch.tuning()[0],
                                   "ms_per_launch": {str(k): round(v, 4) for k, v in arm.batch.tuning()[1].items()}}
                                  if arm.batch is not None else None)}
        errs = []
        for i, d in enumerate(insts):
            Z = _recovered(d, Xs[i])
            if Z is not None and "M" in d.meta:
                M = d.meta["M"]
                errs.append(float(np.linalg.norm(Z - M) / np.linalg.norm(M)))
        if errs:
            line["max_rel_err_vs_planted_M"] = max(errs)
        if ref_arm is not None and arm is not ref_arm:
            eo = [abs(a["obj_p"] - b["obj_p"]) / max(abs(b["obj_p"]), 1e-300) for a, b in zip(res, ref_arm.res)]
            ez = []
            for i, d in enumerate(insts):
                Za, Zb = _recovered(d, Xs[i]), _recovered(d, ref_X[i])
                if Za is None:
                    Za, Zb = Xs[i], ref_X[i]
                ez.append(float(np.linalg.norm(Za - Zb) / max(np.linalg.norm(Zb), 1e-300)))
            line["max_rel_obj_err_vs_fp64"] = max(eo)
            line["max_rel_Z_err_vs_fp64"] = max(ez)
        arm_lines[arm.prec] = line

    # ---- instrumented steps: kernel classes, phases and rooflines
    roof, rooflines, breakdown = None, {}, {}
    if rank == 0 and args.timed_kernel:
        bs = torch.cuda.Stream()
        for prec in dict.fromkeys(precs):
            rep, wall = instrumented_step(args, insts, prec, kk, bs)
            breakdown[prec] = {k: round(v[0], 3) for k, v in sorted(rep.items(), key=lambda kv: -kv[1][0])}
            for cls in ("matvec_b", "matvec_lp_b", "gemm_f64", "potrf", "sytrd", "trsm"):
                r = roofline_of(cls, rep, wall)
                if r is not None:
                    rooflines[f"{prec}:{cls}"] = r
        want = args.timed_kernel if args.timed_kernel != "auto" else "matvec_b"
        roof = rooflines.get(f"fp64:{want}") or next(iter(rooflines.values()), None)
        if roof is not None and roof["kernel"] == "matvec_b" and args.workload == "batched" and args.batch == 16:
            # DRAM bytes of one all-active batched matvec of these 16 instances (ncu
            # captures: SpMM 36.8 MB, SDDMM 37.0 MB; the V assembly is not captured),
            # scaled to the average launch by the flops it did
            t_all, f_all = MATVEC_B_NCU_BYTES, MATVEC_B_ALL_ACTIVE_FLOPS
            per_launch_flops = roof["achieved"] * 1e12 * roof["avg_us"] * 1e-6
            roof["traffic"] = t_all * per_launch_flops / f_all
            roof["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of kb_spmm + kb_sddmm with all "
                                      "16 problems active (profiles/ncu_batched_spmm_16mc.md, "
                                      "profiles/ncu_batched_sddmm_16mc.md), scaled by the average launch's flops")

    # ---- end to end through the public API: host triplets in, solution out (headline arm)
    e2e = None
    if rank == 0 and args.e2e_steps > 0:
        e2e = run_e2e(args, insts, head)

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rate, sample, used = oracle_sample(insts)
        cpu = {"value": rate, "unit": UNIT, "cores": _cores(), "kind": "oracle", "sample": sample,
               "instances": used}

    if rank == 0:
        hl = arm_lines[head.prec]
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": per_arm[head.prec] / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": DTYPES.get(head.prec, head.prec), "data": "synthetic",
                "config": {"workload": desc, "instances": len(insts), "form": FORMS.get(head.prec, head.prec),
                           "arms": precs, "pcg_loop": "graph" if args.pcg_graph else "host",
                           "batched_launch": bool(args.batched_launch),
                           "batch_groups": args.batch_groups if args.batched_launch else None,
                           "parallelism": f"replicas{ws}", "l2_flush": True,
                           "k_max": args.k_max, "eta": args.eta,
                           "inner_rtol_lp": head.params.inner_rtol_lp},
                "latency_ms": {"p50": hl["latency_ms"]["p50"], "p99": hl["latency_ms"]["p99"]},
                "arms": arm_lines,
                "roofline": roof, "rooflines": rooflines or None, "breakdown_ms_per_step": breakdown or None,
                "cpu_baseline": cpu, "e2e": e2e, "clocks": clk.summary(),
                "gpu_launches": int(sum(launches.values()))}
        print(json.dumps(line), flush=True)
    for arm in arms:
        arm.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_e2e(args, insts, head):
    """The headline arm end to end through the public API: host triplets ->
    sdp_setup -> batched (or per-stream) solve -> X and y copied back to the host."""
    import ctypes as C
    import torch
    from paper_1703_10973_gb300 import SDPBatch, SDPProblem
    h2d = sum(d.Ci.nbytes + d.Cj.nbytes + d.Cv.nbytes + d.Ak.nbytes + d.Ai.nbytes + d.Aj.nbytes +
              d.Av.nbytes + d.b.nbytes for d in insts)
    d2h = sum(8 * (d.n * d.n + d.m) for d in insts)
    outs = [(np.empty((d.n, d.n)), np.empty(d.m)) for d in insts]
    torch.cuda.synchronize()
    te = time.perf_counter()
    from concurrent.futures import ThreadPoolExecutor

    def setup(i):   # host-side set-up of each problem in its own thread (the C call releases the GIL)
        return SDPProblem.from_data(insts[i], params=head.params, stream=head.streams[i % len(head.streams)].cuda_stream)

    pool = ThreadPoolExecutor(max_workers=min(16, len(insts)))
    for _ in range(args.e2e_steps):
        ps = list(pool.map(setup, range(len(insts))))
        if args.batched_launch:
            with SDPBatch(ps, stream=head.bstream.cuda_stream, groups=args.batch_groups) as b2:
                b2.solve(allow_maxit=True)
        else:
            errs = []

            def w(s):
                try:
                    for i in range(s, len(ps), len(head.streams)):
                        ps[i].solve(allow_maxit=True)
                except Exception as e:
                    errs.append(e)

            th = [threading.Thread(target=w, args=(s,)) for s in range(len(head.streams))]
            for t in th:
                t.start()
            for t in th:
                t.join()
            if errs:
                raise errs[0]
        def fetch(i):
            X, y = outs[i]
            st = ps[i].lib.sdp_get_solution(ps[i].h, C.c_void_p(X.ctypes.data), C.c_void_p(y.ctypes.data), None)
            assert st == 0
            ps[i].close()

        list(pool.map(fetch, range(len(ps))))
    torch.cuda.synchronize()
    el = time.perf_counter() - te
    pool.shutdown()
    return {"value": args.e2e_steps * len(insts) / el, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h)}


def run_serving(args):
    """Poisson request stream (the serving specs: p, q log-uniform in [50, 3000], r in
    1..5), served by continuous batching (BatchServer: requests join running lockstep
    batches at IPM-iteration boundaries and share every batched PCG launch), with
    admission by a device-memory budget.  Each arm (--arms) first serves every
    request at t = 0 (its capacity), then the arrival rate is swept as fractions of
    that capacity.  Under torchrun each rank serves the requests with rid % world ==
    rank; the line reports rank 0's requests and the whole job's completions."""
    import torch
    import sdp_inputs as si
    from paper_1703_10973_gb300 import _build, default_params, load
    from paper_1703_10973_gb300.serve import BatchServer, Request
    ws, rank, local = _dist()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if not os.path.exists(_build.LIB):
        _build.build()
    load()
    specs = [s for s in si.serving_specs(2000) if s["p"] + s["q"] <= args.serve_max_n][:args.requests]
    insts = [si.mc_instance(s["p"], s["q"], s["r"], s["m"], s["seed"]) for s in specs]
    free, total = torch.cuda.mem_get_info()
    budget = int(0.8 * free)
    precs = [x for x in args.arms.split(",") if x]
    arms, head_cap = {}, None
    with Clocks(local) as clk:
        for prec in precs:
            extra = {"inner_rtol_lp": args.inner_lp} if args.inner_lp > 0 else {}
            params = default_params(prec=prec, pcg_maxit=args.pcg_maxit, **extra)

            def once(arrivals):
                srv = BatchServer(budget_bytes=budget, groups=args.batch_groups or 4, params=params, rank=rank,
                                  world=ws)
                res = srv.run([Request(rid=i, data=d, arrival=float(a))
                               for i, (d, a) in enumerate(zip(insts, arrivals))])
                return srv.stats, res

            once([0.0] * len(insts))   # warm-up: module load, first allocations, graph captures
            cap_stats, cap_res = once([0.0] * len(insts))
            cap = cap_stats["solves_per_s"]
            done = cap_stats["completed"]
            if dist is not None:
                cap = max_over_ranks(-cap, dist, "cuda") * -1.0   # the slowest rank's rate
            sweep = [dict(rate="all at t=0", **{k: cap_stats[k] for k in ("solves_per_s", "p50_ms", "p99_ms",
                                                                           "max_concurrent")})]
            for f in [float(x) for x in args.rates.split(",") if x]:
                rate = f * cap_stats["solves_per_s"] * ws
                st, _ = once(si.serving_arrivals(len(insts), rate))
                sweep.append(dict(rate=rate, rate_frac=f, **{k: st[k] for k in ("solves_per_s", "p50_ms", "p99_ms",
                                                                                 "max_concurrent")}))
            arms[prec] = {"value": cap * ws, "unit": UNIT, "latency_ms": {"p50": cap_stats["p50_ms"],
                                                                          "p99": cap_stats["p99_ms"]},
                          "converged": all(r.converged for r in cap_res if r.ok), "completed_rank0": done,
                          "lockstep_steps": cap_stats["lockstep_steps"], "sweep": sweep,
                          "obj": {r.rid: r.obj_p for r in cap_res if r.ok}}
            if head_cap is None:
                head_cap = arms[prec]["value"]
    ref = arms.get("fp64")
    for prec, a in arms.items():
        if ref is not None and a is not ref:
            a["max_rel_obj_err_vs_fp64"] = max(abs(a["obj"][i] - ref["obj"][i]) / abs(ref["obj"][i])
                                               for i in a["obj"] if i in ref["obj"])
    for a in arms.values():
        a.pop("obj")
    if rank == 0:
        head = arms[precs[0]]
        line = {"metric": METRIC, "value": head_cap, "unit": UNIT, "n_gpus": ws, "steps": len(head["sweep"]),
                "warmup": 1, "ms_per_step": 1e3 * len(insts) / head_cap if head_cap else None,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": DTYPES.get(precs[0], precs[0]), "data": "synthetic",
                "config": {"workload": f"serving: the first {len(insts)} of the 2000 served requests with n <= "
                                       f"{args.serve_max_n} (p, q log-uniform in [50, 3000], r in 1..5, seeds 5000+), "
                                       f"continuous batching in {args.batch_groups or 4} lockstep groups",
                           "form": FORMS.get(precs[0], precs[0]), "arms": precs, "budget_bytes": budget,
                           "parallelism": f"replicas{ws}", "routing": "rid % world == rank"},
                "latency_ms": head["latency_ms"], "arms": arms, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_fig1(args):
    """The paper's Fig. 1 shapes: matrix completion with k = 1 (rank-1 planted M,
    p = q = n / 2) and m = 25 n or m = 0.025 n^2 observations, n swept up to
    --fig1-max-n; per shape, a few interior-point iterations from the start point
    are timed and the median seconds per iteration reported (the quantity Fig. 1
    plots), with the PCG iterations they took."""
    import torch
    import sdp_inputs as si
    from paper_1703_10973_gb300 import SDPProblem, _build, default_params, load
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if not os.path.exists(_build.LIB):
        _build.build()
    load()
    sizes = [n for n in (500, 1000, 2000, 3000, 4000, 5024) if n <= args.fig1_max_n]
    precs = [x for x in args.arms.split(",") if x]
    rows = []
    with Clocks(local) as clk:
        for n in sizes:
            p = n // 2
            for shape, m in (("m=25n", 25 * n), ("m=0.025n^2", int(round(0.025 * n * n)))):
                m = min(m, p * (n - p))
                d = si.mc_instance(p, n - p, 1, m, 7000 + n)
                for prec in precs:
                    params = default_params(prec=prec, pcg_maxit=args.pcg_maxit)
                    with SDPProblem.from_data(d, params=params) as prob:
                        times, pcg = [], []
                        for it in range(args.fig1_iters + 1):
                            torch.cuda.synchronize()
                            t0 = time.perf_counter()
                            info = prob.ipm_step()
                            torch.cuda.synchronize()
                            if it > 0:   # the first iteration includes the first allocations
                                times.append(time.perf_counter() - t0)
                                pcg.append(info["pcg_iters_pred"] + info["pcg_iters_corr"])
                            if info["converged"]:
                                break
                    rows.append(dict(n=n, m=m, shape=shape, prec=prec, s_per_ipm_iter=statistics.median(times),
                                     pcg_iters_per_ipm_iter=float(np.mean(pcg)), iters_timed=len(times)))
                    print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    if rank == 0:
        big = rows[-1]
        line = {"metric": "seconds per interior-point iteration (Fig. 1 shapes)", "value": big["s_per_ipm_iter"],
                "unit": "s", "n_gpus": ws, "steps": args.fig1_iters, "warmup": 1,
                "ms_per_step": 1e3 * big["s_per_ipm_iter"], "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": DTYPES.get(precs[0], precs[0]), "data": "synthetic",
                "config": {"workload": "matrix completion, rank 1, p = q = n/2, m = 25n and m = 0.025n^2 "
                                       f"(the paper's Fig. 1 shapes), n in {sizes}; value: the largest shape",
                           "arms": precs},
                "sweep": rows, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    return 0


def run_probe(args):
    """Small fixed cases for profilers (one JSON line each, timed with CUDA events):
    --probe tc     sdp_mixed_gemm on N x N x N random operands (--probe-n), BF16 then TF32;
    --probe batch  the 16 bench instances joined to an empty batch (sdp_batch_add),
                   --ipm-steps lockstep IPM iterations (sdp_batch_step), host-driven PCG;
    --probe ipm    --ipm-steps IPM iterations of the largest bench instance (B0) alone."""
    import ctypes as C
    import torch
    import sdp_inputs as si
    from paper_1703_10973_gb300 import SDPBatch, SDPProblem, _build, default_params, load
    from paper_1703_10973_gb300 import _lib as L
    _, rank, local = _dist()
    torch.cuda.set_device(local)
    if not os.path.exists(_build.LIB):
        _build.build()
    lib = load()
    out = {"probe": args.probe}
    if args.probe == "tc":
        N = args.probe_n
        for prec in ("bf16", "fp32"):
            A = torch.randn(N, N, dtype=torch.float64, device="cuda")
            B = torch.randn(N, N, dtype=torch.float64, device="cuda")
            Cm = torch.empty(N, N, dtype=torch.float64, device="cuda")
            wb = int(lib.sdp_mixed_gemm_work_bytes(N, N, N))
            work = torch.empty(wb, dtype=torch.uint8, device="cuda")
            err = torch.zeros(1, dtype=torch.int32, device="cuda")
            call = (L.PREC[prec], N, N, N, C.c_void_p(A.data_ptr()), N, 0, C.c_void_p(B.data_ptr()), N, 0,
                    C.c_void_p(Cm.data_ptr()), N, C.c_void_p(work.data_ptr()), wb, C.c_void_p(err.data_ptr()),
                    C.c_void_p(torch.cuda.current_stream().cuda_stream))
            for _ in range(2):
                assert lib.sdp_mixed_gemm(*call) == L.SDP_OK
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(5):
                lib.sdp_mixed_gemm(*call)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 5
            ref = A @ B
            out[prec] = {"ms_per_call": ms, "tflops_incl_packing": 2 * N ** 3 / (ms * 1e-3) / 1e12,
                         "max_rel_err": float((Cm - ref).abs().max() / ref.abs().max()), "flag": int(err.item())}
    elif args.probe == "batch":
        insts, desc = workload("batched", args.batch)
        prm = default_params(pcg_graph=args.pcg_graph, prec=args.arms.split(",")[0])
        streams = [torch.cuda.Stream() for _ in insts]
        probs = [SDPProblem.from_data(d, params=prm, stream=s.cuda_stream) for d, s in zip(insts, streams)]
        b = SDPBatch([])
        for p in probs:
            b.add(p)
        t0 = time.perf_counter()
        for _ in range(args.ipm_steps):
            b.step()
        torch.cuda.synchronize()
        out.update(workload=desc, seconds=time.perf_counter() - t0, tuning=b.tuning()[0])
        b.close()
        for p in probs:
            p.close()
    else:
        s0 = si.batched_specs(256)[0]
        d = si.mc_instance(s0["p"], s0["q"], s0["r"], s0["m"], s0["seed"])
        with SDPProblem.from_data(d, params=default_params(pcg_graph=args.pcg_graph)) as p:
            t0 = time.perf_counter()
            for _ in range(args.ipm_steps):
                p.ipm_step()
            torch.cuda.synchronize()
            out.update(workload=f"B0 (n={d.n}, m={d.m})", seconds=time.perf_counter() - t0)
    if rank == 0:
        print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="batched", choices=["batched", "C2", "C3", "fig2", "fig1", "serving",
                                                              "probe"])
    ap.add_argument("--probe", default="tc", choices=["tc", "batch", "ipm"],
                    help="probe workload: a small fixed case for profilers")
    ap.add_argument("--probe-n", type=int, default=2048, help="probe tc: GEMM order")
    ap.add_argument("--ipm-steps", type=int, default=2, help="probe batch / ipm: interior-point iterations")
    ap.add_argument("--fig1-max-n", type=int, default=5024, help="fig1: largest SDP order of the sweep")
    ap.add_argument("--fig1-iters", type=int, default=3, help="fig1: timed interior-point iterations per shape")
    ap.add_argument("--arms", default="fp32,fp64",
                    help="precision forms timed on the same instances; the first is the headline value")
    ap.add_argument("--k", type=int, default=0, help="split rank (0 = the instance's planted rank)")
    ap.add_argument("--k-max", type=int, default=0, help="adaptive split rank: largest k~ (0 = fixed k)")
    ap.add_argument("--eta", type=float, default=0.0, help="adaptive split rank: eigenvalue-gap ratio")
    ap.add_argument("--inner-lp", type=float, default=0.0,
                    help="PCG tolerance of one reduced-precision sweep (0 = the library default)")
    ap.add_argument("--requests", type=int, default=24, help="serving: requests per arrival rate")
    ap.add_argument("--serve-max-n", type=int, default=800, help="serving: largest SDP order admitted to the sample")
    ap.add_argument("--rates", default="0.25,0.5,1,1.5", help="serving: arrival rates as fractions of capacity")
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--streams", type=int, default=4)
    ap.add_argument("--pcg-maxit", type=int, default=2000)
    ap.add_argument("--timed-kernel", default="auto",
                    help="kernel class of the roofline object (auto = matvec_b, the batched FP64 matvec); "
                         "empty = no instrumented step")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-groups", type=int, default=0,
                    help="lockstep groups solved concurrently (batched mode; 0 = pairs)")
    ap.add_argument("--batched-launch", type=int, default=1, choices=[0, 1],
                    help="1: solve the batch in lockstep with one launch per PCG step for all problems; "
                         "0: independent problems on --streams streams")
    ap.add_argument("--pcg-graph", type=int, default=1, choices=[0, 1],
                    help="0: host-driven PCG loop (same kernels; for profilers without conditional-graph support)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "fig1":
        return run_fig1(args)
    if args.workload == "probe":
        return run_probe(args)
    return run(args)


if __name__ == "__main__":
    sys.exit(main())
