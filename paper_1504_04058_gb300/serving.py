"""Continuous-batching solve server over the C ABI.

Requests (a velocity with an id, omega, grid size, PML/layer widths and a batch
of right-hand sides) arrive at any time.  The server

* keeps factored preconditioners resident in a cache keyed by
  (velocity id, n, omega, PML, b, precision) and evicts the least recently used
  idle entry when a new one does not fit the device-memory budget (admission by
  ``asp_footprint_bytes``);
* batches queued requests that share a cache key into one multi-right-hand-side
  FGMRES solve (up to the handle's ``max_rhs``) -- every right-hand side keeps
  its own Krylov space, so a result does not depend on what it was batched with
  beyond rounding;
* runs several such solves at once on separate CUDA streams (one worker thread
  per stream), so requests that arrive while others are on the GPU start as soon
  as a worker and memory are free;
* records each request's latency from arrival to its solution being on the host.

All compute runs in libasp's kernels; this module only schedules.
"""
from __future__ import annotations

import collections
import dataclasses
import threading
import time
from concurrent.futures import Future

import numpy as np

from . import asp_footprint_bytes, asp_setup, make_params


@dataclasses.dataclass(eq=False)
class Request:
    """One solve request.  ``c`` is the n x n float64 velocity, ``f`` the
    complex128 right-hand sides of shape (n, n, k) (host arrays)."""

    velocity_id: object
    c: np.ndarray
    omega: float
    pml: int
    b: int
    f: np.ndarray
    tol: float = 1e-6
    precision: str = "c64"
    t_arrival: float = 0.0
    rid: int = 0

    @property
    def n(self) -> int:
        return int(self.c.shape[0])

    @property
    def nrhs(self) -> int:
        return int(self.f.shape[-1])

    def key(self):
        return (self.velocity_id, self.n, round(self.omega, 12), self.pml, self.b, self.precision)


@dataclasses.dataclass
class Result:
    rid: int
    u: np.ndarray
    iterations: list
    rel_res_true: list
    latency_s: float
    batched_with: int  # right-hand sides in the solve this request was part of
    factored: bool  # this request's solve had to factor first


class _Entry:
    def __init__(self, handle, footprint, max_rhs):
        self.handle = handle
        self.footprint = footprint
        self.max_rhs = max_rhs
        self.busy = False
        self.last_used = time.monotonic()


class Server:
    """Continuous-batching server.  ``memory_budget`` bytes of device memory are
    available for resident handles; ``workers`` solves may run concurrently."""

    def __init__(self, memory_budget: int, workers: int = 2, max_rhs: int = 8, restart: int = 20,
                 device: int = 0, batching: bool = True, start: bool = True):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.memory_budget = int(memory_budget)
        self.max_rhs = max_rhs
        self.restart = restart
        self.lock = threading.Condition()
        self.queue: collections.deque = collections.deque()
        self.cache: dict = {}
        self.used_bytes = 0
        self.stop = False
        self.batching = batching
        self.active = 0
        self.fatal: BaseException | None = None  # a worker could not start
        self.stats = {"factorizations": 0, "evictions": 0, "solves": 0, "rhs": 0, "max_concurrent": 0}
        self.threads = [threading.Thread(target=self._worker, daemon=True) for _ in range(workers)]
        self.started = False
        if start:
            self.start()

    # ------------------------------------------------------------- public
    def start(self):
        """Start the workers (a server built with ``start=False`` only queues)."""
        if not self.started:
            self.started = True
            for t in self.threads:
                t.start()

    def submit(self, req: Request) -> Future:
        fut: Future = Future()
        if req.t_arrival == 0.0:
            req.t_arrival = time.monotonic()
        with self.lock:
            if self.fatal is not None:
                fut.set_exception(self.fatal)
                return fut
            self.queue.append((req, fut))
            self.lock.notify_all()
        return fut

    def close(self):
        with self.lock:
            self.stop = True
            self.lock.notify_all()
        if self.started:
            for t in self.threads:
                t.join()
        for e in self.cache.values():
            if e.handle is not None:
                e.handle.destroy()
        self.cache.clear()
        self.used_bytes = 0

    # ------------------------------------------------------------ internals
    def _params(self, req: Request):
        return make_params(req.n, req.omega, req.pml, req.b, precision=req.precision,
                           max_rhs=self.max_rhs, restart=self.restart)

    def _admit(self, req: Request):
        """Reserve memory for a new cache entry, evicting idle LRU entries.
        Called with the lock held; returns the footprint or None if it cannot
        fit now (all candidates busy)."""
        fp = asp_footprint_bytes(self._params(req))
        if fp == 0:
            raise ValueError(f"request parameters are invalid or unsupported (n={req.n}, pml={req.pml}, b={req.b}; "
                             "2D takes padded layer widths up to 64 columns and n up to 1216 on 152 SMs)")
        if fp > self.memory_budget:
            raise MemoryError(f"request needs {fp} bytes, budget is {self.memory_budget}")
        while self.used_bytes + fp > self.memory_budget:
            idle = [(e.last_used, k) for k, e in self.cache.items() if not e.busy]
            if not idle:
                return None
            _, k = min(idle)
            e = self.cache.pop(k)
            if e.handle is not None:
                e.handle.destroy()
            self.used_bytes -= e.footprint
            self.stats["evictions"] += 1
        self.used_bytes += fp
        return fp

    def _take_batch(self):
        """Pick the oldest request whose key is not busy, plus (when batching)
        later queued requests with the same key while the batch stays within
        max_rhs right-hand sides.  A request wider than max_rhs runs alone and
        is solved in chunks.  Lock held."""
        for idx, (req, _) in enumerate(self.queue):
            k = req.key()
            e = self.cache.get(k)
            if e is not None and e.busy:
                continue
            batch, total = [self.queue[idx]], req.nrhs
            if self.batching:
                for item in list(self.queue)[idx + 1:]:
                    r2 = item[0]
                    if r2.key() == k and total + r2.nrhs <= self.max_rhs:
                        batch.append(item)
                        total += r2.nrhs
            for item in batch:
                self.queue.remove(item)
            return k, batch
        return None, None

    def _worker(self):
        torch = self.torch
        try:
            torch.cuda.set_device(self.device)
            stream = torch.cuda.Stream(device=self.device)
        except BaseException as ex:  # no usable device: fail what is queued and what comes
            with self.lock:
                self.fatal = ex
                while self.queue:
                    _, fut = self.queue.popleft()
                    fut.set_exception(ex)
                self.lock.notify_all()
            return
        while True:
            with self.lock:
                while True:
                    if self.stop and not self.queue:
                        return
                    k, batch = self._take_batch()
                    if batch is not None:
                        e = self.cache.get(k)
                        factored = False
                        if e is None:
                            fp = self._admit(batch[0][0])
                            if fp is None:  # no memory right now: put back and wait
                                for item in reversed(batch):
                                    self.queue.appendleft(item)
                                self.lock.wait(timeout=0.01)
                                continue
                            e = _Entry(None, fp, self.max_rhs)
                            self.cache[k] = e
                            factored = True
                        e.busy = True
                        self.active += 1
                        self.stats["max_concurrent"] = max(self.stats["max_concurrent"], self.active)
                        break
                    self.lock.wait(timeout=0.05)
            try:
                self._run(e, batch, stream, factored)
            except BaseException as ex:  # report to every future of the batch
                for _, fut in batch:
                    if not fut.done():
                        fut.set_exception(ex)
                with self.lock:
                    if e.handle is None:
                        self.cache.pop(k, None)
                        self.used_bytes -= e.footprint
            finally:
                with self.lock:
                    self.active -= 1
                    e.busy = False
                    e.last_used = time.monotonic()
                    self.lock.notify_all()

    def _run(self, e: _Entry, batch, stream, factored: bool):
        torch = self.torch
        req0 = batch[0][0]
        with torch.cuda.stream(stream):
            if e.handle is None:
                e.handle = asp_setup(req0.c, self._params(req0))
                e.handle.factor(stream=stream)
                with self.lock:
                    self.stats["factorizations"] += 1
            f = np.concatenate([r.f for r, _ in batch], axis=-1)
            fd = torch.from_numpy(np.ascontiguousarray(f)).pin_memory().to(self.device, non_blocking=True)
            tol = min(r.tol for r, _ in batch)
            parts, info = [], []
            for c0 in range(0, f.shape[-1], self.max_rhs):
                u, inf = e.handle.gmres_solve(fd[..., c0:c0 + self.max_rhs].contiguous(), tol=tol, maxit=400,
                                              stream=stream, raise_on_nonconvergence=False)
                parts.append(u)
                info += inf
            uh = torch.cat(parts, dim=-1).to("cpu", non_blocking=True)
            stream.synchronize()
        uh = uh.numpy()
        t_done = time.monotonic()
        total = f.shape[-1]
        with self.lock:
            self.stats["solves"] += 1
            self.stats["rhs"] += total
        col = 0
        for r, fut in batch:
            k = r.nrhs
            res = Result(r.rid, uh[..., col:col + k].copy(), [i["iterations"] for i in info[col:col + k]],
                         [i["rel_res_true"] for i in info[col:col + k]], t_done - r.t_arrival, total, factored)
            col += k
            fut.set_result(res)


def percentiles(latencies, qs=(50, 99)):
    arr = np.sort(np.asarray(latencies))
    return {f"p{q}": float(np.percentile(arr, q)) for q in qs}


def run_stream(requests, memory_budget: int, workers: int = 2, max_rhs: int = 8, restart: int = 20,
               realtime: bool = True, precision: str = "c64", batching: bool = True):
    """Replay requests (dicts from workloads.serving_stream) through a Server,
    each submitted at its arrival time ``t`` (seconds after the start) when
    ``realtime``, else all at once; returns (results, wall seconds, stats)."""
    import workloads as W
    srv = Server(memory_budget, workers=workers, max_rhs=max_rhs, restart=restart, batching=batching)
    futs = []
    t0 = time.monotonic()
    for i, d in enumerate(requests):
        if realtime:
            delay = t0 + d["t"] - time.monotonic()
            if delay > 0:
                time.sleep(delay)
        P = W.materialize(d)
        req = Request(("layered", d["velocity_seed"]), P.c, P.omega, P.pml, P.b, P.f, tol=P.tol,
                      precision=precision, rid=i)
        futs.append(srv.submit(req))
    results = [f.result() for f in futs]
    wall = time.monotonic() - t0
    stats = dict(srv.stats)
    srv.close()
    return results, wall, stats


def main():
    import argparse
    import json

    import workloads as W
    ap = argparse.ArgumentParser(description="serving stream: Poisson-arriving 2D requests")
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--sizes", default="255,511")
    ap.add_argument("--rate", type=float, default=50.0, help="mean arrivals per second")
    ap.add_argument("--velocity-pool", type=int, default=8)
    ap.add_argument("--budget-gb", type=float, default=120.0)
    ap.add_argument("--workers", type=int, default=2)
    ap.add_argument("--max-rhs", type=int, default=16)
    ap.add_argument("--capacity", action="store_true",
                    help="submit every request at once (measures the sustainable request rate)")
    ap.add_argument("--one-at-a-time", action="store_true",
                    help="baseline: complex128 factors, one request per solve, no cache reuse across keys")
    args = ap.parse_args()
    sizes = tuple(int(s) for s in args.sizes.split(","))
    reqs = W.serving_stream(args.requests, rate_hz=args.rate, sizes=sizes, velocity_pool=args.velocity_pool)
    if args.one_at_a_time:
        results, wall, stats = run_stream(reqs, int(args.budget_gb * 2**30), workers=1, max_rhs=8,
                                          realtime=False, precision="c128", batching=False)
    else:
        results, wall, stats = run_stream(reqs, int(args.budget_gb * 2**30), workers=args.workers,
                                          max_rhs=args.max_rhs, realtime=not args.capacity)
    lat = [r.latency_s for r in results]
    nrhs = sum(len(r.iterations) for r in results)
    out = {"requests": len(results), "rhs": nrhs, "wall_s": wall, "solves_per_s": nrhs / wall,
           "requests_per_s": len(results) / wall,
           **{k: v for k, v in percentiles(lat).items()}, "stats": stats,
           "worst_rel_res_true": max(max(r.rel_res_true) for r in results)}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
