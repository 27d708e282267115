"""Serving loops: SDP requests arriving over time on one GPU.

BatchServer (continuous batching).  Admitted requests join running lockstep
batches (sdp_batch_add) at interior-point iteration boundaries and leave them
when they finish (sdp_batch_remove): every PCG iteration of all the members'
Newton systems is one sequence of batched launches, so a request that arrives
while others run shares their kernels from its first iteration on.  ``groups``
batches run concurrently, each driven by its own host thread, so that one
group's dense phases overlap another's batched PCG; an admitted request joins
the group with the least work in flight.

Server (one resident problem per slot).  Each admitted request is solved on its
own by one of ``slots`` CUDA streams (``sdp_setup`` ... ``sdp_solve`` ...
``sdp_destroy``); requests overlap but do not share launches.

Both admit first come, first served, gated by a device-memory budget: a request
is started only when the estimated bytes of every problem in flight plus its own
fit the budget (a request larger than the whole budget is rejected).  Finished
problems release their bytes at once.  Requests with rid % world != rank are
left to the other ranks (one server per GPU, no exchange between them).

The admission logic is plain host code; the solvers are callables or CUDA
handles, so the rules can be exercised without a GPU.
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


def _latency_stats(out, extra):
    done = [r for r in out if r.ok]
    lat = sorted(r.latency for r in done)
    span = (max(r.finish for r in done) - min(r.arrival for r in done)) if done else 0.0
    stats = dict(completed=len(done), rejected=len(out) - len(done),
                 solves_per_s=(len(done) / span) if span > 0 else 0.0,
                 p50_ms=1e3 * lat[len(lat) // 2] if lat else math.nan,
                 p99_ms=1e3 * lat[min(len(lat) - 1, int(math.ceil(0.99 * len(lat))) - 1)] if lat else math.nan)
    stats.update(extra)
    return stats


@dataclass
class BatchServer:
    """Continuous batching of requests into lockstep batches (see the module docstring)."""
    budget_bytes: int
    groups: int = 4
    params: object = None          # sdp_params of every request (precision, tolerances)
    keep_solution: bool = False
    rank: int = 0
    world: int = 1
    stats: dict = field(default_factory=dict)

    def run(self, requests: list[Request]) -> list[Result]:
        import torch
        from .api import SDPBatch, SDPProblem
        mine = [r for r in requests if r.rid % self.world == self.rank]
        for r in mine:
            if not r.est_bytes:
                r.est_bytes = estimate_request_bytes(r.data)
        pending = sorted(mine, key=lambda r: (r.arrival, r.rid))
        lock = threading.Condition()
        G = max(1, self.groups)
        state = dict(in_flight=0, max_in_flight=0, members=[0] * G, work=[0] * G, max_members=0, done=0,
                     steps=0, arrived_all=False, abort=False)
        inbox = [[] for _ in range(G)]
        results: dict[int, Result] = {}
        t0 = time.perf_counter()
        errors = []

        def group(g):
            bstream = torch.cuda.Stream(priority=-1)   # the batched PCG ahead of other groups' dense phases
            batch = SDPBatch([], stream=bstream.cuda_stream)
            members = {}                     # id(prob) -> (prob, request, start, stream)
            free_streams = []
            try:
                while True:
                    with lock:
                        while not inbox[g] and not members and not state["abort"] and not (
                                state["arrived_all"] and state["done"] >= len(pending)):
                            lock.wait(0.05)
                        if state["abort"] or (not inbox[g] and not members):
                            return
                        joining = inbox[g]
                        inbox[g] = []
                    for req in joining:
                        start = time.perf_counter() - t0
                        st = free_streams.pop() if free_streams else torch.cuda.Stream()
                        try:
                            prob = SDPProblem.from_data(req.data, params=self.params, stream=st.cuda_stream)
                            batch.add(prob)
                            members[id(prob)] = (prob, req, start, st)
                        except Exception as e:
                            self._finish(lock, state, results, g, req, start, t0, error=str(e))
                            free_streams.append(st)
                    if not members:
                        continue
                    batch.step()
                    with lock:
                        state["steps"] += 1
                    for key, (prob, req, start, st) in list(members.items()):
                        res, where, status = batch.member(prob)
                        if where == "running":
                            continue
                        sol = prob.get_solution() if self.keep_solution else None
                        batch.remove(prob)
                        err = "" if where != "failed" else f"status {status}: {prob.lib.sdp_last_error(prob.h).decode()}"
                        dev = prob.device_bytes()
                        prob.close()
                        del members[key]
                        free_streams.append(st)
                        self._finish(lock, state, results, g, req, start, t0, res=res, converged=(where == "converged"),
                                     error=err, solution=sol, device_bytes=dev)
            except Exception as e:  # surfaced after the run; the other groups stop too
                errors.append(e)
                with lock:
                    state["abort"] = True
                    lock.notify_all()
            finally:
                batch.close()

        threads = [threading.Thread(target=group, args=(g,), daemon=True) for g in range(G)]
        for t in threads:
            t.start()
        waiting: list[Request] = []
        i = 0
        with lock:
            while state["done"] < len(pending) and not errors:
                now = time.perf_counter() - t0
                while i < len(pending) and pending[i].arrival <= now:
                    waiting.append(pending[i])
                    i += 1
                while waiting:
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
                    g = min(range(G), key=lambda x: (state["work"][x], state["members"][x]))
                    state["in_flight"] += head.est_bytes
                    state["max_in_flight"] = max(state["max_in_flight"], state["in_flight"])
                    state["members"][g] += 1
                    state["work"][g] += head.est_bytes
                    state["max_members"] = max(state["max_members"], sum(state["members"]))
                    inbox[g].append(head)
                    lock.notify_all()
                if i >= len(pending):
                    state["arrived_all"] = True
                    lock.notify_all()
                if state["done"] >= len(pending):
                    break
                timeout = 1.0
                if i < len(pending):
                    timeout = max(0.0, pending[i].arrival - (time.perf_counter() - t0))
                lock.wait(timeout=min(timeout, 1.0))
            state["arrived_all"] = True
            if errors:
                state["abort"] = True
            lock.notify_all()
        for t in threads:
            t.join()
        if errors:
            raise errors[0]
        out = [results[r.rid] for r in sorted(mine, key=lambda r: r.rid)]
        self.stats = _latency_stats(out, dict(max_in_flight_bytes=state["max_in_flight"],
                                              max_concurrent=state["max_members"], budget_bytes=self.budget_bytes,
                                              groups=G, lockstep_steps=state["steps"]))
        return out

    @staticmethod
    def _finish(lock, state, results, g, req, start, t0, res=None, converged=False, error="", solution=None,
                device_bytes=0):
        now = time.perf_counter() - t0
        r = Result(rid=req.rid, ok=(res is not None and not error), arrival=req.arrival, start=start, finish=now,
                   error=error, solution=solution, device_bytes=device_bytes)
        if res is not None:
            r.converged = converged
            r.obj_p = res["obj_p"]
            r.relgap = res["relgap"]
            r.iters = res["iters"]
        with lock:
            results[req.rid] = r
            state["in_flight"] -= req.est_bytes
            state["members"][g] -= 1
            state["work"][g] -= req.est_bytes
            state["done"] += 1
            lock.notify_all()
