"""Continuous-batching solve service over the C ABI.

Requests (an MDP in host memory plus solve options) arrive over time.  A
request is admitted as soon as one of `slots` workers is free and its device
footprint fits in what is left of the HBM budget; each worker owns a CUDA
stream, uploads the MDP (mdp_create), runs Algorithm 1 (mdp_solve) and copies
V and the policy back, so admitted requests overlap on the GPU while later
ones wait.  With batch_max > 1 a worker takes, besides the first request that
fits, later pending requests that also fit (any S, A, k and gamma; GMRES in
FP64 or mixed precision) and solves them together with mdp_solve_batch: one launch per pass for
all of them, each result bit for bit its stand-alone one.  With small_states > 0, requests of at most that
many states (GMRES in FP64) are instead gathered with the other pending small ones, up to small_batch_max,
and solved by mdp_solve_small_batch: one thread-block cluster per request, the whole batch in one launch
(solve_alone routes such a request the same way, so each result is still bit for bit its stand-alone
one).  With graph set (the default), every grid solve runs graph-driven (opts.graph): a single
request as one CUDA graph launch, a batch as one graph whose branches are its members' solves, with
no host round trip until they stop; the results are the same bit for bit as stream-driven solves.
The solver calls release the Python interpreter lock, so the
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
    # an MDPData-like object (S, A, row_ptr, col, val, g, gamma as host arrays), or
    # one with S, A, gamma, nnz, kmax and device_arrays() -> (row_ptr, col, val, g)
    # device tensors made when a worker admits the request (on the worker's stream)
    data: object
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
    error: str = ""  # the library's message when status is not MDP_OK

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def device_bytes(data, restart: int = 30, precision: int = mdp.MDP_PREC_F64) -> int:
    """Upper estimate of a request's device footprint: the stacked matrix in the
    sliced layout (12 B per entry), what mdp_create holds besides it, the policy
    rows, costs, work vectors and the Krylov basis."""
    S, A = int(data.S), int(data.A)
    if hasattr(data, "device_arrays"):  # drawn on the device at admission: sizes known up front
        nnz, kmax = int(data.nnz), int(data.kmax)
        return _footprint(S, A, nnz, kmax, restart, precision, host=False)
    nnz = int(data.row_ptr[-1])
    kmax = int(np.max(np.diff(data.row_ptr))) if S * A else 0
    return _footprint(S, A, nnz, kmax, restart, precision, host=True)


# mdp_create uploads host entries in row-aligned chunks of at most this many entries
# (or one longest row), through at most four device buffers
UPLOAD_CHUNK_ENTRIES = 1 << 25
UPLOAD_BUFFERS = 4


def _creation_bytes(S, A, nnz, kmax, host) -> int:
    """Device memory mdp_create holds besides the handle: the row pointers and row
    lengths, and either the upload's chunk buffers (host input: each chunk but the last
    holds more than cap - kmax entries, so their number is bounded) or the request's
    own device copy of the CSR (device input, until mdp_create returns)."""
    rows = 8 * (S * A + 1) + 4 * S * A
    if not host:
        return rows + 12 * nnz
    cap = min(nnz, max(UPLOAD_CHUNK_ENTRIES, kmax))
    chunks = 1 if nnz <= cap else nnz // max(1, cap - kmax + 1) + 1
    return rows + 12 * cap * min(UPLOAD_BUFFERS, chunks)


def _footprint(S, A, nnz, kmax, restart, precision, host=True) -> int:
    stacked = 12 * nnz + 8 * S * A
    upload = _creation_bytes(S, A, nnz, kmax, host)
    policy = 16 * S * kmax
    basis = 8 * (restart + 1) * S + (4 * (restart + 1) * S if precision == mdp.MDP_PREC_MIXED else 0)
    vectors = 16 * 8 * S
    return stacked + upload + policy + basis + vectors + (1 << 20)


def _create(d, stream):
    """mdp_create from host arrays, or from device arrays the request makes now."""
    if hasattr(d, "device_arrays"):
        rp, col, val, g = d.device_arrays()
        out = mdp.mdp_create(d.S, d.A, rp, col, val, g, True, stream)  # copies; returns after the copy
        del rp, col, val, g
        return out
    return mdp.mdp_create(d.S, d.A, d.row_ptr, d.col, d.val, d.g, False, stream)


class SolveService:
    """A fixed pool of worker slots with an HBM admission budget."""

    def __init__(self, slots: int = 4, hbm_budget: int = 120 << 30, device: int = 0, batch_max: int = 1,
                 keep=None, small_states: int = 0, small_batch_max: int = 256, graph: bool = True):
        """keep: optional predicate on a request id; results of other requests drop V and
        the policy (status, iteration counts and latency stay), to bound host memory on
        long streams."""
        import torch
        self.slots = slots
        self.batch_max = max(1, int(batch_max))
        self.small_states = int(small_states)
        self.small_batch_max = max(1, int(small_batch_max))
        self.graph = bool(graph)
        self.keep = keep
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
        self.batches: list[int] = []  # size of every solve the workers ran
        self.oom_retries = 0  # requests requeued after running out of device memory
        self._retry_wait = False  # hold admissions until a request in flight finishes

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
    @staticmethod
    def _batchable(r: Request) -> bool:
        return r.inner == mdp.MDP_GMRES and r.precision in (mdp.MDP_PREC_F64, mdp.MDP_PREC_MIXED)

    def _small(self, r: Request) -> bool:
        return is_small(r, self.small_states)

    def _admit(self):
        """First pending request (arrival order) that fits the free budget, plus (with
        batch_max > 1) later pending requests that still fit, when all of them run
        GMRES: they are solved together by one mdp_solve_batch call."""
        for i, r in enumerate(self._pending):
            need = device_bytes(r.data, r.restart, r.precision)
            if need <= self._free:
                batch = [r]
                total = need
                if self._small(r):  # small requests go together to the cluster solver
                    for r2 in self._pending[i + 1:]:
                        if len(batch) == self.small_batch_max:
                            break
                        n2 = device_bytes(r2.data, r2.restart, r2.precision)
                        if self._small(r2) and total + n2 <= self._free:
                            batch.append(r2)
                            total += n2
                elif self.batch_max > 1 and self._batchable(r):
                    for r2 in self._pending[i + 1:]:
                        if len(batch) == self.batch_max:
                            break
                        n2 = device_bytes(r2.data, r2.restart, r2.precision)
                        if self._batchable(r2) and total + n2 <= self._free:
                            batch.append(r2)
                            total += n2
                ids = {id(b) for b in batch}
                self._pending = [p for p in self._pending if id(p) not in ids]
                self._free -= total
                return batch, total
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
                    batch, need = (None, 0) if self._retry_wait else self._admit()
                    if batch is not None:
                        break
                    self._cv.wait()
                self._in_flight += len(batch)
                self.peak_in_flight = max(self.peak_in_flight, self._in_flight)
            admitted = self.now()
            retry = False
            try:
                if self._small(batch[0]):
                    outs = self._solve_small(batch, stream)
                elif len(batch) == 1:
                    outs = [self._solve(batch[0], stream, self.graph)]
                else:
                    outs = self._solve_batch(batch, stream, self.graph)
            except Exception as exc:  # failed requests still complete, with their status
                status = exc.status if isinstance(exc, mdp.MDPError) else mdp.MDP_ERR_CUDA
                oom = isinstance(exc, torch.cuda.OutOfMemoryError) or status == mdp.MDP_ERR_OOM
                outs = [Result(r.rid, status if not oom else mdp.MDP_ERR_OOM, np.empty(0),
                               np.empty(0, dtype=np.int32), 0, 0, float("nan"), r.arrival, 0.0, 0.0, str(exc))
                        for r in batch]
                retry = oom
                if oom:
                    torch.cuda.empty_cache()  # hand torch's unused cached blocks back before the retry
            finally:
                with self._cv:
                    self._free += need
                    self._in_flight -= len(batch)
                    # the budget is an estimate (caching allocators, fragmentation): a request that
                    # ran out of device memory while others were in flight goes back to the front
                    # of the queue and is admitted again once one of them finishes
                    if retry and self._in_flight > 0:
                        self._pending[0:0] = batch
                        self.oom_retries += len(batch)
                        self._retry_wait = True
                    else:
                        retry = False
                    self._cv.notify_all()
            if retry:
                continue
            done = self.now()
            with self._cv:
                self._retry_wait = False
                for res in outs:
                    res.admitted = admitted
                    res.finished = done
                    if self.keep is not None and not self.keep(res.rid):
                        res.V, res.pi = np.empty(0), np.empty(0, dtype=np.int32)
                    self._results[res.rid] = res
                self.batches.append(len(batch))
                self._cv.notify_all()

    @staticmethod
    def _solve(req: Request, stream, graph: bool = True) -> Result:
        import torch
        d = req.data
        with torch.cuda.stream(stream):
            st, h = _create(d, stream)
            mdp.check(st, f"mdp_create (request {req.rid})")
            try:
                o = mdp.mdp_default_opts()
                o.gamma, o.atol_pi, o.alpha, o.inner = d.gamma, req.tol, req.alpha, req.inner
                o.gmres_restart, o.precision, o.graph = req.restart, req.precision, int(graph)
                V = torch.zeros(d.S, dtype=torch.float64, device="cuda")
                pi = torch.empty(d.S, dtype=torch.int32, device="cuda")
                st, stats = mdp.mdp_solve(h, o, V, pi, stream)
                err = mdp.mdp_last_error() if st != mdp.MDP_OK else ""
                Vh, pih = V.cpu(), pi.cpu()  # on this stream: ordered after the solve
            finally:
                mdp.mdp_destroy(h)
        return Result(req.rid, st, Vh.numpy(), pih.numpy(), stats.outer_iters, int(stats.inner_iters_total),
                      stats.final_residual, req.arrival, 0.0, 0.0, err)

    @staticmethod
    def _solve_batch(batch, stream, graph: bool = True) -> list:
        import torch
        handles = []
        with torch.cuda.stream(stream):
            try:
                for r in batch:
                    st, h = _create(r.data, stream)
                    mdp.check(st, f"mdp_create (request {r.rid})")
                    handles.append(h)
                opts = []
                for r in batch:
                    o = mdp.mdp_default_opts()
                    o.gamma, o.atol_pi, o.alpha, o.inner = r.data.gamma, r.tol, r.alpha, r.inner
                    o.gmres_restart, o.precision, o.graph = r.restart, r.precision, int(graph)
                    opts.append(o)
                V = [torch.zeros(r.data.S, dtype=torch.float64, device="cuda") for r in batch]
                pi = [torch.empty(r.data.S, dtype=torch.int32, device="cuda") for r in batch]
                st, status, stats = mdp.mdp_solve_batch(handles, opts, V, pi, stream)
                mdp.check(st, "mdp_solve_batch")
                Vh = [v.cpu() for v in V]  # on this stream: ordered after the solve
                pih = [p.cpu() for p in pi]
            finally:
                for h in handles:
                    mdp.mdp_destroy(h)
        return [Result(r.rid, status[i], Vh[i].numpy(), pih[i].numpy(), stats[i].outer_iters,
                       int(stats[i].inner_iters_total), stats[i].final_residual, r.arrival, 0.0, 0.0)
                for i, r in enumerate(batch)]


    @staticmethod
    def _solve_small(batch, stream) -> list:
        import torch
        handles = []
        with torch.cuda.stream(stream):
            try:
                for r in batch:
                    st, h = _create(r.data, stream)
                    mdp.check(st, f"mdp_create (request {r.rid})")
                    handles.append(h)
                opts = []
                for r in batch:
                    o = mdp.mdp_default_opts()
                    o.gamma, o.atol_pi, o.alpha, o.inner = r.data.gamma, r.tol, r.alpha, r.inner
                    o.gmres_restart, o.precision = r.restart, r.precision
                    opts.append(o)
                V = [torch.zeros(r.data.S, dtype=torch.float64, device="cuda") for r in batch]
                pi = [torch.empty(r.data.S, dtype=torch.int32, device="cuda") for r in batch]
                st, status, stats = mdp.mdp_solve_small_batch(handles, opts, V, pi, stream)
                mdp.check(st, "mdp_solve_small_batch")
                Vh = [v.cpu() for v in V]  # on this stream: ordered after the solve
                pih = [p.cpu() for p in pi]
            finally:
                for h in handles:
                    mdp.mdp_destroy(h)
        return [Result(r.rid, status[i], Vh[i].numpy(), pih[i].numpy(), stats[i].outer_iters,
                       int(stats[i].inner_iters_total), stats[i].final_residual, r.arrival, 0.0, 0.0)
                for i, r in enumerate(batch)]


def is_small(r: Request, small_states: int) -> bool:
    """Whether the cluster solver takes the request: at most small_states (and 65,536) states,
    GMRES in FP64."""
    return (0 < int(r.data.S) <= min(small_states, 65536) and r.inner == mdp.MDP_GMRES
            and r.precision == mdp.MDP_PREC_F64)


def solve_alone(req: Request, small_states: int = 0, graph: bool = True) -> Result:
    """The same request on the current stream with nothing else running (routed to the
    cluster solver, as a service with the same small_states would, when it is small;
    graph- or stream-driven otherwise)."""
    import torch
    t0 = time.perf_counter()
    if is_small(req, small_states):
        res = SolveService._solve_small([req], torch.cuda.current_stream())[0]
    else:
        res = SolveService._solve(req, torch.cuda.current_stream(), graph)
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
