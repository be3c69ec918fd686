"""Continuous-batching solve service over the C ABI.

Requests (an MDP in host memory plus solve options) arrive over time.  A
request is admitted as soon as one of `slots` workers is free and its device
footprint fits in what is left of the HBM budget; each worker owns a CUDA
stream, uploads the MDP (mdp_create), runs Algorithm 1 (mdp_solve) and copies
V and the policy back, so admitted requests overlap on the GPU while later
ones wait.  The solver calls release the Python interpreter lock, so the
workers' host threads run concurrently.  All computation happens in libmdp's
kernels; this module only schedules.
"""
from __future__ import annotations

import dataclasses
import threading
import time

import numpy as np

from . import mdp


@dataclasses.dataclass
class Request:
    rid: int
    data: object  # an MDPData-like object: S, A, row_ptr, col, val, g, gamma
    tol: float = 1e-8
    alpha: float = 1e-3
    inner: int = mdp.MDP_GMRES
    restart: int = 30
    precision: int = mdp.MDP_PREC_F64
    arrival: float = 0.0  # seconds after the service started


@dataclasses.dataclass
class Result:
    rid: int
    status: int
    V: np.ndarray
    pi: np.ndarray
    outer_iters: int
    inner_iters: int
    final_residual: float
    arrival: float
    admitted: float
    finished: float

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def device_bytes(data, restart: int = 30, precision: int = mdp.MDP_PREC_F64) -> int:
    """Upper estimate of a request's device footprint: the stacked matrix in the
    sliced layout (12 B per entry), its temporary CSR copy during upload, the
    policy rows, costs, work vectors and the Krylov basis."""
    S, A = int(data.S), int(data.A)
    nnz = int(data.row_ptr[-1])
    kmax = int(np.max(np.diff(data.row_ptr))) if S * A else 0
    stacked = 12 * nnz + 8 * S * A
    upload = 12 * nnz + 8 * (S * A + 1)
    policy = 16 * S * kmax
    basis = 8 * (restart + 1) * S + (4 * (restart + 1) * S if precision == mdp.MDP_PREC_MIXED else 0)
    vectors = 16 * 8 * S
    return stacked + upload + policy + basis + vectors + (1 << 20)


class SolveService:
    """A fixed pool of worker slots with an HBM admission budget."""

    def __init__(self, slots: int = 4, hbm_budget: int = 120 << 30, device: int = 0):
        import torch
        self.slots = slots
        self.budget = int(hbm_budget)
        self.device = device
        self._free = self.budget
        self._cv = threading.Condition()
        self._pending: list[Request] = []
        self._results: dict[int, Result] = {}
        self._stop = False
        self._t0 = None
        mdp.load()
        self._streams = [torch.cuda.Stream(device=device) for _ in range(slots)]
        self._workers = [threading.Thread(target=self._work, args=(i,), daemon=True) for i in range(slots)]
        self.peak_in_flight = 0
        self._in_flight = 0

    # -- client side --------------------------------------------------------------
    def start(self):
        self._t0 = time.perf_counter()
        for w in self._workers:
            w.start()
        return self

    def now(self) -> float:
        return time.perf_counter() - self._t0

    def submit(self, req: Request):
        need = device_bytes(req.data, req.restart, req.precision)
        if need > self.budget:
            raise ValueError(f"request {req.rid} needs {need} bytes, above the whole budget {self.budget}")
        with self._cv:
            req.arrival = self.now()
            self._pending.append(req)
            self._cv.notify_all()

    def close(self):
        with self._cv:
            self._stop = True
            self._cv.notify_all()
        for w in self._workers:
            w.join()

    def results(self) -> dict:
        with self._cv:
            return dict(self._results)

    def wait(self, n: int, timeout: float = 600.0) -> dict:
        end = time.perf_counter() + timeout
        with self._cv:
            while len(self._results) < n:
                left = end - time.perf_counter()
                if left <= 0:
                    raise TimeoutError(f"{len(self._results)} of {n} requests finished")
                self._cv.wait(left)
            return dict(self._results)

    # -- workers ------------------------------------------------------------------
    def _admit(self):
        """First pending request (arrival order) that fits the free budget."""
        for i, r in enumerate(self._pending):
            need = device_bytes(r.data, r.restart, r.precision)
            if need <= self._free:
                self._free -= need
                return self._pending.pop(i), need
        return None, 0

    def _work(self, slot: int):
        import torch
        torch.cuda.set_device(self.device)
        stream = self._streams[slot]
        while True:
            with self._cv:
                while True:
                    if self._stop and not self._pending:
                        return
                    req, need = self._admit()
                    if req is not None:
                        break
                    self._cv.wait()
                self._in_flight += 1
                self.peak_in_flight = max(self.peak_in_flight, self._in_flight)
            admitted = self.now()
            try:
                res = self._solve(req, stream)
            except Exception as exc:  # a failed request still completes, with its status
                status = exc.status if isinstance(exc, mdp.MDPError) else mdp.MDP_ERR_CUDA
                res = Result(req.rid, status, np.empty(0), np.empty(0, dtype=np.int32), 0, 0, float("nan"),
                             req.arrival, 0.0, 0.0)
            finally:
                with self._cv:
                    self._free += need
                    self._in_flight -= 1
                    self._cv.notify_all()
            res.admitted = admitted
            res.finished = self.now()
            with self._cv:
                self._results[req.rid] = res
                self._cv.notify_all()

    @staticmethod
    def _solve(req: Request, stream) -> Result:
        import torch
        d = req.data
        with torch.cuda.stream(stream):
            st, h = mdp.mdp_create(d.S, d.A, d.row_ptr, d.col, d.val, d.g, False, stream)
            mdp.check(st, f"mdp_create (request {req.rid})")
            try:
                o = mdp.mdp_default_opts()
                o.gamma, o.atol_pi, o.alpha, o.inner = d.gamma, req.tol, req.alpha, req.inner
                o.gmres_restart, o.precision = req.restart, req.precision
                V = torch.zeros(d.S, dtype=torch.float64, device="cuda")
                pi = torch.empty(d.S, dtype=torch.int32, device="cuda")
                st, stats = mdp.mdp_solve(h, o, V, pi, stream)
                Vh, pih = V.cpu(), pi.cpu()  # on this stream: ordered after the solve
            finally:
                mdp.mdp_destroy(h)
        return Result(req.rid, st, Vh.numpy(), pih.numpy(), stats.outer_iters, int(stats.inner_iters_total),
                      stats.final_residual, req.arrival, 0.0, 0.0)


def solve_alone(req: Request) -> Result:
    """The same request on the current stream with nothing else running."""
    import torch
    t0 = time.perf_counter()
    res = SolveService._solve(req, torch.cuda.current_stream())
    res.finished = time.perf_counter() - t0
    return res


def latency_summary(results: dict) -> dict:
    lat = np.array([r.latency for r in results.values()])
    span = max(r.finished for r in results.values()) - min(r.arrival for r in results.values())
    return {"requests": len(lat), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "solves_per_s": len(lat) / span if span > 0 else None, "span_s": span}


def fifo_one_at_a_time(arrivals, service_times) -> dict:
    """Latencies of the same arrivals served one request at a time in arrival order
    (start = max(arrival, previous finish)), from measured stand-alone solve times."""
    t = 0.0
    lat = []
    for a, d in zip(arrivals, service_times):
        t = max(t, a) + d
        lat.append(t - a)
    lat = np.array(lat)
    span = t - min(arrivals)
    return {"requests": len(lat), "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_s": float(lat.mean()), "solves_per_s": len(lat) / span if span > 0 else None, "span_s": span}
