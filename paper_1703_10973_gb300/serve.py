"""Serving loop: SDP requests arriving over time, continuous batching on one GPU.

Each admitted request becomes one resident problem (``sdp_setup`` ... ``sdp_solve``
... ``sdp_destroy``) on one of ``slots`` CUDA streams, so requests that arrive
while others are on the GPU overlap with them.  Admission is first come, first
served, gated by a device-memory budget: a request is started only when a slot
is free and the estimated bytes of every problem in flight plus its own fit the
budget (a request larger than the whole budget is rejected).  Finished problems
release their slot and their bytes at once.

The scheduler is plain host logic; the solver is a callable, so the admission
rules can be exercised without a GPU.
"""
from __future__ import annotations

import math
import queue
import threading
import time
from dataclasses import dataclass, field


def estimate_bytes(n: int, m: int, k: int, r_side: int | None = None) -> int:
    """Upper estimate of the device bytes of one resident problem (FP64, Hhat).

    About 31 dense n x n FP64 arrays (iterate, NT scaling, step-length inverses,
    eigensolver workspace), the two dense Schur-complement factors of order
    r_side * k (r_side: rows outside the independent set; n / 2 when unknown),
    O(n k) preconditioner vectors, O(m) PCG vectors and constraint structure,
    and a fixed allowance.
    """
    rk = (r_side if r_side is not None else (n + 1) // 2) * k
    return int(8 * (31 * n * n + 2 * rk * rk + 8 * n * k + 1000 * n) + 220 * m + (8 << 20))


def estimate_request_bytes(d) -> int:
    """estimate_bytes for an SDPData; matrix-completion instances give their smaller side."""
    meta = getattr(d, "meta", None) or {}
    r_side = None
    if "p" in meta and "q" in meta:
        r_side = min(int(meta["p"]), int(meta["q"]))
    return estimate_bytes(d.n, d.m, d.k, r_side)


@dataclass
class Request:
    rid: int
    data: object
    arrival: float          # seconds after the start of the run
    est_bytes: int = 0


@dataclass
class Result:
    rid: int
    ok: bool
    converged: bool = False
    obj_p: float = math.nan
    relgap: float = math.nan
    iters: int = 0
    arrival: float = 0.0
    start: float = 0.0
    finish: float = 0.0
    device_bytes: int = 0
    error: str = ""
    solution: tuple | None = None

    @property
    def latency(self) -> float:
        return self.finish - self.arrival


def cuda_solver(params=None, keep_solution=False):
    """Solver callable for Server: one resident problem per request on `stream`."""
    from .api import SDPProblem

    def solve(d, stream):
        with SDPProblem.from_data(d, params=params, stream=stream) as prob:
            res = prob.solve(allow_maxit=True)
            out = dict(converged=bool(res["converged"]), obj_p=res["obj_p"], relgap=res["relgap"],
                       iters=res["iters"], device_bytes=prob.device_bytes())
            if keep_solution:
                out["solution"] = prob.get_solution()
            return out
    return solve


@dataclass
class Server:
    budget_bytes: int
    slots: int = 8
    solver: object = None          # callable(data, stream) -> dict; default: the CUDA solve
    make_stream: object = None     # callable() -> stream handle for a slot (default: a torch stream)
    stats: dict = field(default_factory=dict)

    def run(self, requests: list[Request]) -> list[Result]:
        solver = self.solver if self.solver is not None else cuda_solver()
        streams = self._streams()
        for r in requests:
            if not r.est_bytes:
                r.est_bytes = estimate_request_bytes(r.data)
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        lock = threading.Condition()
        state = dict(in_flight=0, busy=0, max_in_flight=0, max_busy=0, done=0)
        results: dict[int, Result] = {}
        work = [queue.Queue() for _ in range(self.slots)]
        free = list(range(self.slots))
        t0 = time.perf_counter()

        def worker(s):
            while True:
                req = work[s].get()
                if req is None:
                    return
                start = time.perf_counter() - t0
                try:
                    out = solver(req.data, streams[s])
                    res = Result(rid=req.rid, ok=True, arrival=req.arrival, start=start, **{
                        k: v for k, v in out.items() if k in ("converged", "obj_p", "relgap", "iters",
                                                              "device_bytes", "solution")})
                except Exception as e:  # reported in the result, the server keeps going
                    res = Result(rid=req.rid, ok=False, arrival=req.arrival, start=start, error=str(e))
                res.finish = time.perf_counter() - t0
                with lock:
                    results[req.rid] = res
                    state["in_flight"] -= req.est_bytes
                    state["busy"] -= 1
                    state["done"] += 1
                    free.append(s)
                    lock.notify_all()

        threads = [threading.Thread(target=worker, args=(s,), daemon=True) for s in range(self.slots)]
        for t in threads:
            t.start()
        waiting: list[Request] = []
        i = 0
        with lock:
            while state["done"] < len(pending):
                now = time.perf_counter() - t0
                while i < len(pending) and pending[i].arrival <= now:
                    waiting.append(pending[i])
                    i += 1
                # first come, first served: the head waits for room, later requests wait behind it
                while waiting and free:
                    head = waiting[0]
                    if head.est_bytes > self.budget_bytes:
                        waiting.pop(0)
                        results[head.rid] = Result(rid=head.rid, ok=False, arrival=head.arrival, start=now,
                                                   finish=now, error="larger than the memory budget")
                        state["done"] += 1
                        continue
                    if state["in_flight"] + head.est_bytes > self.budget_bytes:
                        break
                    waiting.pop(0)
                    s = free.pop(0)
                    state["in_flight"] += head.est_bytes
                    state["busy"] += 1
                    state["max_in_flight"] = max(state["max_in_flight"], state["in_flight"])
                    state["max_busy"] = max(state["max_busy"], state["busy"])
                    work[s].put(head)
                if state["done"] >= len(pending):
                    break
                timeout = None
                if i < len(pending):
                    timeout = max(0.0, pending[i].arrival - (time.perf_counter() - t0))
                lock.wait(timeout=timeout if timeout is not None else 1.0)
        for q in work:
            q.put(None)
        for t in threads:
            t.join()
        out = [results[r.rid] for r in sorted(requests, key=lambda r: r.rid)]
        done = [r for r in out if r.ok]
        lat = sorted(r.latency for r in done)
        span = (max(r.finish for r in done) - min(r.arrival for r in done)) if done else 0.0
        self.stats = dict(
            completed=len(done), rejected=len(out) - len(done),
            solves_per_s=(len(done) / span) if span > 0 else 0.0,
            p50_ms=1e3 * lat[len(lat) // 2] if lat else math.nan,
            p99_ms=1e3 * lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)] if lat else math.nan,
            max_in_flight_bytes=state["max_in_flight"], max_concurrent=state["max_busy"],
            budget_bytes=self.budget_bytes, slots=self.slots)
        return out

    def _streams(self):
        if self.make_stream is not None:
            return [self.make_stream() for _ in range(self.slots)]
        try:
            import torch
            if torch.cuda.is_available():
                return [torch.cuda.Stream().cuda_stream for _ in range(self.slots)]
        except Exception:
            pass
        return [None] * self.slots
