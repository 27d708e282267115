"""Benchmark: SDP solves/s and per-solve latency at 1e-6 relative duality gap.

Default workload ("batched"): the first 16 instances of the batched
matrix-completion workload (p, q uniform in [50, 400], r uniform in {1..4},
m = min(pq/2, ceil(3 r (p+q) ln(p+q))) uniform observations, seeds 4000..4015).
One step solves all 16 SDPs, each from the interior-point start point to
relative gap, primal and dual infeasibility <= 1e-6 with every Newton system
solved by PCG to a 1e-8 true relative residual.  By default the 16 problems are
advanced in lockstep (sdp_batch_solve): their dense phases on one stream and
host thread each, and every PCG iteration of all 16 Newton systems as one
sequence of batched launches under a CUDA graph.  --batched-launch 0 solves
them as independent problems on --streams streams.  The problem data stay in
HBM across steps; each solve resets its iterate on the device.

`--workload C2` runs the single n = 1000, m = 8000, rank-2 instance instead; its
nuclear-norm optimum has rank about 38, outside the low-rank regime the
preconditioner is built for, and PCG stalls before 1e-6 (the line reports it).

The printed line (rank 0) carries the contract keys plus: latency_ms (p50/p99
per solve), roofline (dominant kernel class, timed with CUDA events over one
instrumented step after the timed ones), cpu_baseline (the FP64 oracle on the
host cores, bounded sample), e2e (host triplets -> sdp_setup -> solve ->
solution copied back, through the public API), clocks (nvidia-smi samples taken
during the timed region) and gpu_launches (library kernels in the timed region).

--impl reference times the FP64 oracle (explicit Hessian + Cholesky) on the host
cores on a bounded sample of the same workload.  Under torchrun (--gpus N) each
rank solves its own 16 instances (ranks take distinct blocks of the 256) with no
collective on the data path; the step time is the maximum over ranks.
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

METRIC = "SDP solves/s at 1e-6 relative duality gap"
UNIT = "solves/s"

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
        return [d], ("matrix-completion SDP n1=n2=500 (n=1000), rank 2, m=8000, seed 2; "
                     "plain method, k=8 (optimum rank ~38)")
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


def cpu_oracle_rate(insts, iters_per_solve, budget_s=25.0):
    """Oracle IPM iterations on the batch's instances (smallest first) for ~budget_s."""
    from oracle import sdp_oracle as o
    done_t, done_i, used = 0.0, 0, []
    for d in sorted(insts, key=lambda d: d.m):
        P = o.Problem.from_data(d)
        t0 = time.perf_counter()
        o.ipm_solve(P, o.IPMParams(maxit=1))
        el = time.perf_counter() - t0
        done_t += el
        done_i += 1
        used.append((d.n, d.m, el))
        if done_t > budget_s:
            break
    # scale: mean oracle seconds per IPM iteration over the sampled instances (weighted
    # to the batch by m^3, the Cholesky cost) times iterations per solve
    w_s = sum(el for _, _, el in used)
    w_m = sum(m ** 3 for _, m, _ in used)
    all_m = sum(d.m ** 3 for d in insts)
    est_batch_iter = w_s * all_m / w_m
    solve_s = est_batch_iter * iters_per_solve
    sample = (f"one oracle IPM iteration (explicit m x m Hessian + Cholesky, NumPy/LAPACK FP64) on "
              f"{done_i} of the {len(insts)} instances ({w_s:.1f} s), extrapolated to the batch by m^3 and "
              f"to {iters_per_solve:.1f} IPM iterations per solve")
    return len(insts) / solve_s, sample


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    insts, desc = workload(args.workload, args.batch)
    times = []
    from oracle import sdp_oracle as o
    small = sorted(insts, key=lambda d: d.m)[0]
    P = o.Problem.from_data(small)
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        o.ipm_solve(P, o.IPMParams(maxit=1))
        if step >= args.warmup:
            times.append(time.perf_counter() - t0)
    per_iter_small = statistics.median(times)
    scale = sum(d.m ** 3 for d in insts) / small.m ** 3
    iters = 20.0
    value = len(insts) / (per_iter_small * scale * iters)
    sample = (f"one oracle IPM iteration on the smallest instance (n={small.n}, m={small.m}) per step, "
              f"scaled to the batch by m^3 and to {iters:.0f} IPM iterations per solve")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * len(insts) / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": desc, "instances": len(insts), "l2_flush": False},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": _cores(), "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run(args):
    import torch
    ws, rank, local = _dist()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1703_10973_gb300 import SDPProblem, _build, default_params, load
    if not os.path.exists(_build.LIB):
        _build.build()
    load()
    insts, desc = workload(args.workload, args.batch, rank, ws)
    kk = 8 if args.workload == "C2" else 0
    params = default_params(prec=args.prec, k=kk, pcg_maxit=args.pcg_maxit, pcg_graph=args.pcg_graph)
    nstreams = len(insts) if args.batched_launch else min(args.streams, len(insts))
    streams = [torch.cuda.Stream() for _ in range(nstreams)]
    probs = [SDPProblem.from_data(d, params=params, stream=streams[i % nstreams].cuda_stream)
             for i, d in enumerate(insts)]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    batch = None
    stage_ms = {}          # batched mode: wall ms per lockstep stage of the last solve
    if args.batched_launch:
        from paper_1703_10973_gb300 import SDPBatch
        bstream = torch.cuda.Stream()
        batch = SDPBatch(probs, stream=bstream.cuda_stream, groups=args.batch_groups)

    def run_batch(start_event=None):
        """Solve every instance once; stream s handles instances s, s+S, ...  Returns per-solve ms."""
        if batch is not None:   # lockstep: one launch per PCG step for all problems
            if start_event is not None:
                bstream.wait_event(start_event)
                for st in streams:
                    st.wait_event(start_event)
            torch.cuda.synchronize()
            for p in probs:
                p.reset()
            t0b = time.perf_counter()
            res_b = batch.solve(allow_maxit=True)
            torch.cuda.synchronize()
            ms = (time.perf_counter() - t0b) * 1e3
            stage_ms.update({k: (round(v * 1e3, 1) if k not in ("graph_launches", "batched_iters") else int(v))
                             for k, v in batch.stage_seconds().items()})
            return [ms] * len(probs), res_b
        if start_event is not None:
            for st in streams:
                st.wait_event(start_event)
        lat = [None] * len(probs)
        res = [None] * len(probs)
        errs = []

        def worker(s):
            try:
                st = streams[s]
                for i in range(s, len(probs), nstreams):
                    a = torch.cuda.Event(enable_timing=True)
                    b = torch.cuda.Event(enable_timing=True)
                    a.record(st)
                    probs[i].reset()
                    res[i] = probs[i].solve(allow_maxit=True)
                    b.record(st)
                    b.synchronize()
                    lat[i] = a.elapsed_time(b)
            except Exception as e:  # surfaced after join
                errs.append(e)

        th = [threading.Thread(target=worker, args=(s,)) for s in range(nstreams)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        if errs:
            raise errs[0]
        return lat, res

    for _ in range(args.warmup):
        run_batch()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    l0 = probs[0].launch_count()
    step_ms, lat_all, res_last = [], [], None
    with Clocks(local) as clk:
        for i in range(args.steps):
            flush.fill_(float(i))          # evict L2 between steps (256 MB > 126 MB L2)
            torch.cuda.synchronize()
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record()
            lat, res = run_batch(t0)
            for s in streams:              # join every stream into the default stream
                torch.cuda.current_stream().wait_stream(s)
            t1.record()
            torch.cuda.synchronize()
            step_ms.append(t0.elapsed_time(t1))
            lat_all += lat
            res_last = res
    launches = probs[0].launch_count() - l0
    stage_timed = dict(stage_ms)
    total_ms = sum(step_ms)
    if dist is not None:
        total_ms = max_over_ranks(total_ms, dist, "cuda")
        dist.barrier()
    solves = len(insts) * args.steps * ws
    value = solves / (total_ms / 1e3)
    converged = all(r["converged"] for r in res_last)
    ipm_iters = [r["iters"] for r in res_last]
    pcg_iters = [r["pcg_iters_total"] for r in res_last]

    # ---- one instrumented step: CUDA events around every kernel class and phase
    roof, breakdown = None, None
    if rank == 0 and args.timed_kernel:
        if batch is not None:
            # the batched PCG runs inside a graph, whose kernels events cannot
            # bracket: the instrumented step drives the same batched kernels from
            # the host (pcg_graph = 0), all problems in one lockstep group
            from paper_1703_10973_gb300 import SDPBatch, default_params as _dp
            iparams = _dp(prec=args.prec, k=kk, pcg_maxit=args.pcg_maxit, pcg_graph=0)
            iprobs = [SDPProblem.from_data(d, params=iparams, stream=streams[i % nstreams].cuda_stream)
                      for i, d in enumerate(insts)]
            ib = SDPBatch(iprobs, stream=bstream.cuda_stream, groups=1)
            torch.cuda.synchronize()
            iprobs[0].timing_enable("*")
            tk0 = time.perf_counter()
            ib.solve(allow_maxit=True)
            torch.cuda.synchronize()
            step_wall = (time.perf_counter() - tk0) * 1e3
            rep = iprobs[0].timing_report()
            iprobs[0].timing_enable(None)
            ib.close()
            for p in iprobs:
                p.close()
        else:
            probs[0].timing_enable("*")
            tk0 = time.perf_counter()
            run_batch()
            torch.cuda.synchronize()
            step_wall = (time.perf_counter() - tk0) * 1e3
            rep = probs[0].timing_report()
            probs[0].timing_enable(None)
        breakdown = {k: round(v[0], 3) for k, v in sorted(rep.items(), key=lambda kv: -kv[1][0])}
        if args.timed_kernel == "auto":
            # the batched PCG matvec (SpMM + SDDMM of every active problem in one
            # launch each) when the step ran batched: it is the hot path's kernel
            # and, in the lockstep instrumented step, runs with nothing beside it;
            # otherwise the kernel class with the most device time (phases excluded)
            kcls = [k for k in rep if k not in PHASES and rep[k][2] > 0]
            if args.prec == "fp64" and "matvec_b" in kcls and rep["matvec_b"][1] > 0:
                args.timed_kernel = "matvec_b"
            else:
                args.timed_kernel = max(kcls, key=lambda k: rep[k][0]) if kcls else "sytrd"
        kt = rep.get(args.timed_kernel)
        if kt and kt[1]:
            ms, cnt, fl, by = kt
            avg = ms / cnt
            if args.timed_kernel in ALU_CLASSES:
                ach = fl / (ms * 1e-3) / 1e12
                roof = {"kernel": args.timed_kernel, "bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS,
                        "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS, "traffic": None,
                        "peak_source": FP64_PEAK_SOURCE, "launches": cnt, "avg_us": avg * 1e3,
                        "busy_ms_per_step": ms, "step_ms_instrumented": step_wall}
            else:
                peak = _peaks().get("hbm_gbs", 6674.2)
                ach = by / (ms * 1e-3) / 1e9
                roof = {"kernel": args.timed_kernel, "bound": "hbm", "achieved": ach, "peak": peak,
                        "unit": "GB/s", "frac": ach / peak, "traffic": None,
                        "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json)",
                        "fp64_tflops": fl / (ms * 1e-3) / 1e12, "launches": cnt, "avg_us": avg * 1e3,
                        "busy_ms_per_step": ms, "step_ms_instrumented": step_wall}

    # ---- end to end through the public API: host triplets in, solution out
    e2e = None
    if rank == 0 and args.e2e_steps > 0:
        import ctypes as C
        h2d = sum(d.Ci.nbytes + d.Cj.nbytes + d.Cv.nbytes + d.Ak.nbytes + d.Ai.nbytes + d.Aj.nbytes +
                  d.Av.nbytes + d.b.nbytes for d in insts)
        d2h = sum(8 * (d.n * d.n + d.m) for d in insts)
        outs = [(np.empty((d.n, d.n)), np.empty(d.m)) for d in insts]
        torch.cuda.synchronize()
        te = time.perf_counter()
        for _ in range(args.e2e_steps):
            errs = []

            def e2e_worker(s):
                try:
                    for i in range(s, len(insts), nstreams):
                        p2 = SDPProblem.from_data(insts[i], params=params, stream=streams[s].cuda_stream)
                        p2.solve(allow_maxit=True)
                        X, y = outs[i]
                        st = p2.lib.sdp_get_solution(p2.h, C.c_void_p(X.ctypes.data), C.c_void_p(y.ctypes.data),
                                                     None)
                        assert st == 0
                        p2.close()
                except Exception as e:
                    errs.append(e)

            if args.batched_launch:   # set up all, solve in lockstep, copy every solution back
                from paper_1703_10973_gb300 import SDPBatch
                ps = [SDPProblem.from_data(insts[i], params=params, stream=streams[i].cuda_stream)
                      for i in range(len(insts))]
                with SDPBatch(ps, stream=bstream.cuda_stream, groups=args.batch_groups) as b2:
                    b2.solve(allow_maxit=True)
                for i, p2 in enumerate(ps):
                    X, y = outs[i]
                    st = p2.lib.sdp_get_solution(p2.h, C.c_void_p(X.ctypes.data), C.c_void_p(y.ctypes.data), None)
                    assert st == 0
                    p2.close()
                continue
            th = [threading.Thread(target=e2e_worker, args=(s,)) for s in range(nstreams)]
            for t in th:
                t.start()
            for t in th:
                t.join()
            if errs:
                raise errs[0]
        torch.cuda.synchronize()
        el = time.perf_counter() - te
        e2e = {"value": args.e2e_steps * len(insts) / el, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h)}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rate, sample = cpu_oracle_rate(insts, float(np.mean(ipm_iters)))
        cpu = {"value": rate, "unit": UNIT, "cores": _cores(), "kind": "oracle", "sample": sample}

    if rank == 0:
        srt = sorted(lat_all)
        p50 = srt[len(srt) // 2]
        p99 = srt[min(len(srt) - 1, int(math.ceil(0.99 * len(srt))) - 1)]
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.prec == "fp64" else args.prec,
                "data": "synthetic",
                "config": {"workload": desc, "instances": len(insts), "streams": nstreams, "prec": args.prec, "pcg_loop": "graph" if args.pcg_graph else "host",
                           "batched_launch": bool(args.batched_launch),
                           "batch_groups": args.batch_groups if args.batched_launch else None,
                           "parallelism": f"replicas{ws}", "l2_flush": True, "converged": converged,
                           "ipm_iters_mean": float(np.mean(ipm_iters)),
                           "pcg_iters_per_solve_mean": float(np.mean(pcg_iters)),
                           "max_relgap": max(r["relgap"] for r in res_last)},
                "latency_ms": {"p50": p50, "p99": p99},
                "roofline": roof, "stage_ms_per_step": stage_timed or None, "breakdown_ms_per_step": breakdown, "cpu_baseline": cpu, "e2e": e2e,
                "clocks": clk.summary(),
                "gpu_launches": int(launches)}
        print(json.dumps(line), flush=True)
    if batch is not None:
        batch.close()
    for p in probs:
        p.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_serving(args):
    """Poisson request stream (the serving specs: p, q log-uniform, r in 1..5), continuous
    batching with admission by a device-memory budget; the arrival rate is swept as
    fractions of the capacity measured with every request present at time 0."""
    import torch
    import sdp_inputs as si
    from paper_1703_10973_gb300 import _build, load
    from paper_1703_10973_gb300.serve import Request, Server, cuda_solver
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if not os.path.exists(_build.LIB):
        _build.build()
    load()
    specs = [s for s in si.serving_specs(2000) if s["p"] + s["q"] <= args.serve_max_n][:args.requests]
    insts = [si.mc_instance(s["p"], s["q"], s["r"], s["m"], s["seed"]) for s in specs]
    free, total = torch.cuda.mem_get_info()
    budget = int(0.8 * free)
    solver = cuda_solver()

    def once(arrivals):
        srv = Server(budget_bytes=budget, slots=args.streams, solver=solver)
        res = srv.run([Request(rid=i, data=d, arrival=float(a)) for i, (d, a) in enumerate(zip(insts, arrivals))])
        return srv.stats, res

    once([0.0] * len(insts))                         # warm-up (module load, first allocations)
    with Clocks(local) as clk:
        cap_stats, cap_res = once([0.0] * len(insts))
        cap = cap_stats["solves_per_s"]
        sweep = [dict(rate="all at t=0", **{k: cap_stats[k] for k in ("solves_per_s", "p50_ms", "p99_ms",
                                                                       "max_concurrent")})]
        for f in [float(x) for x in args.rates.split(",") if x]:
            rate = f * cap
            arr = si.serving_arrivals(len(insts), rate)
            st, _ = once(arr)
            sweep.append(dict(rate=rate, rate_frac=f, **{k: st[k] for k in ("solves_per_s", "p50_ms", "p99_ms",
                                                                             "max_concurrent")}))
    if rank == 0:
        line = {"metric": METRIC, "value": cap, "unit": UNIT, "n_gpus": ws, "steps": len(sweep),
                "warmup": 1, "ms_per_step": 1e3 * len(insts) / cap if cap else None, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": f"serving: first {len(insts)} of the 2000 served requests with n <= "
                                       f"{args.serve_max_n} (p, q log-uniform in [50, 3000], r in 1..5, seeds 5000+)",
                           "slots": args.streams, "budget_bytes": budget,
                           "converged": all(r.converged for r in cap_res if r.ok),
                           "completed": cap_stats["completed"]},
                "latency_ms": {"p50": cap_stats["p50_ms"], "p99": cap_stats["p99_ms"]},
                "serving_sweep": sweep, "clocks": clk.summary()}
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="batched", choices=["batched", "C2", "serving"])
    ap.add_argument("--requests", type=int, default=24, help="serving: requests per arrival rate")
    ap.add_argument("--serve-max-n", type=int, default=800, help="serving: largest SDP order admitted to the sample")
    ap.add_argument("--rates", default="0.25,0.5,1,1.5", help="serving: arrival rates as fractions of capacity")
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--streams", type=int, default=4)
    ap.add_argument("--prec", default="fp64", choices=["fp64", "fp32", "bf16"])
    ap.add_argument("--pcg-maxit", type=int, default=2000)
    ap.add_argument("--timed-kernel", default="auto",
                    help="kernel class for the roofline object; auto = the batched PCG matvec when the "
                         "step ran batched, else the class with the most device time")
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
    return run(args)


if __name__ == "__main__":
    sys.exit(main())
