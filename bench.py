#!/usr/bin/env python
"""Benchmark: inexact policy iteration to ||TV - V||_inf <= 1e-8 on the banded
epidemic-like MDP (S = 1e6 infected counts, A = 20 intervention levels, 33-wide
binomial bands, gamma = 0.999, GMRES(30), alpha = 0.01), synthetic inputs.

One step = one full mdp_solve from V_0 = 0: every Bellman sweep, policy-row
gather, Arnoldi step (mat-vec and classical Gram-Schmidt) and Givens update of
Algorithm 1 until the stop test holds.  Inputs (8.3 GB) stay resident in HBM and are larger than L2, so no L2
flush is needed between steps.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

With torchrun (N > 1) every rank solves its own replica (the path does not
shard: replicas only); rank 0 prints one JSON line with the max-over-ranks time.
--impl reference times the FP64 CPU oracle instead (rank 0 only).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")  # the CPU oracle runs single-threaded

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("iPI time to ‖TV−V‖∞≤1e-8; Bellman SpMV+min GB/s vs HBM peak; "
          "p50/p99 latency")
S, A, H, GAMMA = 1_000_000, 20, 16, 0.999
K_ROW = 2 * H + 1
TOL, ALPHA, RESTART = 1e-8, 0.01, 30
# FP64 FMA peak of GB300: 152 SMs x 2 FP64 FMA per SM per clock x 2 flops x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def workload_config():
    return {"workload": "banded epidemic-like MDP (SIS-step band centres)", "S": S, "A": A, "k": K_ROW,
            "nnz": S * A * K_ROW, "gamma": GAMMA, "tol": TOL, "alpha": ALPHA, "inner": f"GMRES({RESTART})",
            "V0": "zeros", "l2": "inputs (8.3 GB) larger than L2 (129 MB); no flush"}


def bellman_bytes():
    """Algorithmic bytes of one Bellman sweep: CSR values (8) + columns (4) per
    entry, row pointers (8) and costs (8) per row, V read once, TV and pi written."""
    R = S * A
    nnz = R * K_ROW
    return nnz * 12 + (R + 1) * 8 + R * 8 + S * 8 + S * (8 + 4)




_DGEMM = {}


def fp64_dgemm_tflops(n=4096, reps=5):
    """Measured FP64 rate of this GPU: torch.matmul of two n x n binary64 matrices (cuBLAS
    DGEMM), best of `reps`, 2 n^3 flops each; measured once per process."""
    if "v" not in _DGEMM:
        import torch
        a = torch.rand(n, n, dtype=torch.float64, device="cuda")
        b = torch.rand(n, n, dtype=torch.float64, device="cuda")
        torch.matmul(a, b)
        best = None
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1) * 1e-3
            best = t if best is None else min(best, t)
        _DGEMM["v"] = 2.0 * n ** 3 / best / 1e12
        del a, b
    return _DGEMM["v"]


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def bellman_source_sha():
    """sha256 (first 16 hex digits) of the sources that make the Bellman kernel."""
    h = hashlib.sha256()
    for f in ("sell.cuh", "bellman_dev.cuh", "bellman.cu"):
        h.update(open(os.path.join(ROOT, "paper_2507_22538_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def krylov_source_sha():
    """sha256 (first 16 hex digits) of the code that makes the fused GMRES mat-vec + dots
    kernel: sell.cuh and krylov_dev.cuh (the row layout and the kernel body) and the
    kernel's own definition in krylov.cu (host code there does not change it)."""
    csrc = os.path.join(ROOT, "paper_2507_22538_gb300", "csrc")
    h = hashlib.sha256()
    for f in ("sell.cuh", "krylov_dev.cuh"):
        h.update(open(os.path.join(csrc, f), "rb").read())
    src = open(os.path.join(csrc, "krylov.cu"), "rb").read()
    start = src.index(b"gm_matvec_dots_kernel(const double* __restrict__ pval,")
    start = src.rindex(b"template", 0, start)
    h.update(src[start:src.index(b"\n}\n", start) + 3])
    return h.hexdigest()[:16]


def summary_value(name, key, sha_key, sha):
    """A number from a committed ncu summary under profiles/, if it was taken on the
    current kernel source (else None)."""
    summ = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(summ):
        return None
    vals = {}
    for line in open(summ):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get(sha_key) != sha:
        return None
    try:
        return float(vals[key])
    except (KeyError, ValueError):
        return None


def lowp_bytes(S_, A_, k_):
    """Algorithmic bytes of one low-precision sweep (generic-CSR accounting): 16-bit
    value (2) + column (4) per entry, row pointer (8) and cost (8) per row, V read once,
    TV and pi written.  The binary64 re-evaluation of the candidate rows re-reads them
    while they are still in L2 and is not counted."""
    R = S_ * A_
    return R * k_ * 6 + R * 16 + S_ * 20


def sweep_traffic():
    """DRAM bytes per Bellman launch from the committed ncu summary, if it was taken
    on the current kernel source (else None)."""
    summ = os.path.join(ROOT, "profiles", "bellman_sweep_banded_s1e6.txt")
    if not os.path.exists(summ):
        return None
    sha = bellman_source_sha()
    vals = {}
    for line in open(summ):
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("bellman_src_sha256_16") != sha:
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) >= 9:
                    rows.append(f)
        except OSError:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def max_over_ranks(value, dist=None, device=None):
    """Max of a per-rank float over all ranks (identity without a process group)."""
    if dist is None or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def certified_bound(res, gamma, kmax, gnorm, vnorm):
    """Bound on ||V - V*||_inf from a computed Bellman residual res = ||TV - V||_inf
    (Sec. II: T is a gamma-contraction, so ||V - V*|| <= ||TV - V|| / (1 - gamma)),
    widened by the rounding of the residual's own computation: each Q is a
    length-kmax recursive dot product plus cost, off by at most
    gamma_{k+2} (|g| + gamma |V|) with gamma_n = n u / (1 - n u) (Higham, Sec. 3.1)."""
    u = 2.0 ** -53
    n = kmax + 2
    q = n * u / (1 - n * u) * (gnorm + gamma * vnorm)
    return (res + q) / (1 - gamma)


def error_statement(V, pi, res, gamma, kmax, gnorm, ref=None, ref_name="fp64_gpu"):
    """The error of one solve's result: the certified bound against the exact V*, and
    (when a reference result is given) its distance to it and the policy mismatches."""
    import numpy as np
    vn = float(np.max(np.abs(V)))
    out = {"certified_bound_vs_Vstar": certified_bound(res, gamma, kmax, gnorm, vn),
           "relative_certified_bound": certified_bound(res, gamma, kmax, gnorm, vn) / vn if vn else None}
    if ref is not None:
        rV, rpi = ref
        out[f"max_abs_diff_vs_{ref_name}"] = float(np.max(np.abs(V - rV)))
        out[f"policy_mismatches_vs_{ref_name}"] = int(np.sum(pi != rpi))
    return out


def cpu_info():
    """The host the CPU oracle runs on: logical cores and the CPU model (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model or "unknown"}


def cpu_oracle_solve(save_v=None, states=S, m=None):
    """Time the FP64 oracle's Algorithm 1 on the bench workload itself (S = 1e6, same
    generator, gamma, tol, alpha and GMRES(30)): numpy/scipy with one thread (its
    sparse products are single-threaded scipy; BLAS is pinned to one thread above).
    Returns (seconds, iteration info); optionally saves V and pi (.npz) for the error
    statement of the GPU results."""
    import numpy as np
    from mdpgen import banded_birth_death
    from oracle import mdp_oracle as O
    if m is None:
        m = banded_birth_death(states, A, H, GAMMA)
    t0 = time.perf_counter()
    r = O.ipi(m.S, m.A, m.row_ptr, m.col, m.val, m.g, m.gamma, tol=TOL, alpha=ALPHA, inner="gmres",
              restart=RESTART)
    dt = time.perf_counter() - t0
    if save_v:
        np.savez(save_v, V=r.V, pi=r.pi)
    return dt, {"converged": bool(r.converged), "outer": int(r.outer_iters), "inner": int(sum(r.inner_iters)),
                "final_residual": float(r.residuals[-1])}


def run_cpu_oracle_worker(args):
    """Child process of the bench: waits for a line on stdin (the parent sends it once the
    kernel and end-to-end timings are done, so that the oracle's memory traffic and host
    load stay out of them), then times one oracle solve of the full workload on one host
    core while the remaining GPU measurements proceed; prints one JSON line."""
    if not sys.stdin.readline():  # the parent ended without asking for the solve
        return 0
    t, info = cpu_oracle_solve(save_v=args.cpu_oracle_worker)
    print(json.dumps({"seconds": t, "info": info, **cpu_info()}), flush=True)
    return 0


def cpu_oracle_all_cores():
    """The same oracle solve with its BLAS allowed every host core (run after the GPU
    sections, so it disturbs none of them); scipy's sparse products, most of the solve,
    stay single-threaded, so this is the oracle as it stands with all cores available,
    not a parallelised oracle."""
    nthreads = os.cpu_count() or 1
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = str(nthreads)
    fd, npz = tempfile.mkstemp(suffix=".npz")
    os.close(fd)
    try:
        child = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-oracle-worker", npz], input="go\n",
                               capture_output=True, text=True, env=env, timeout=600)
        rec = json.loads(child.stdout.strip().splitlines()[-1])
        return {"value": rec["seconds"], "unit": "s", "threads": nthreads,
                "note": "BLAS threads = host cores; the sparse products stay single-threaded"}
    except (subprocess.TimeoutExpired, ValueError, IndexError, KeyError) as e:
        return {"value": None, "unit": "s", "threads": nthreads, "note": f"failed: {e}"}
    finally:
        os.unlink(npz)


REFERENCE_BUDGET_S = 150.0  # the reference arm stops timing further solves after this much wall time


def run_reference(args):
    """The FP64 CPU oracle timed on the bench workload itself.  One solve takes 30-100 s
    on one core, so the arm times solves back to back until `steps` are done or
    REFERENCE_BUDGET_S has passed (at least one), runs no warm-up solve (the oracle
    keeps no state between solves), and reports the number it timed as `steps`."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    times, info = [], None
    states = args.reference_states or S
    from mdpgen import banded_birth_death
    m = banded_birth_death(states, A, H, GAMMA)  # the instance, drawn once (outside the timing)
    t_start = time.perf_counter()
    while len(times) < max(1, args.steps):
        t, info = cpu_oracle_solve(states=states, m=m)
        times.append(t)
        if time.perf_counter() - t_start + t > REFERENCE_BUDGET_S:
            break
    v = statistics.median(times)
    host = cpu_info()
    sample = (f"FP64 numpy/scipy oracle, Algorithm 1 with MGS-GMRES(30), on the bench workload itself "
              f"(S={states}, same generator, gamma, tol, alpha), {len(times)} solve(s) timed of {args.steps} requested "
              f"(one solve takes ~{v:.0f} s; the arm stops after {REFERENCE_BUDGET_S:.0f} s), no warm-up; "
              f"one thread on a {host['nproc']}-core {host['cpu_model']} host; last run {info}")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "s", "n_gpus": world,
            "steps": len(times), "warmup": 0, "steps_requested": args.steps, "warmup_requested": args.warmup,
            "ms_per_step": v * 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(workload_config(), S=states, nnz=states * A * K_ROW),
            "cpu_baseline": {"value": v, "unit": "s", "cores": 1, "kind": "oracle", "sample": sample,
                             "runs_s": times, **host},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


class DeviceRequest:
    """A request of the counter-based serving stream, drawn on the device (CUDA
    generator) when a worker admits it: the stand-in for the client's upload."""

    def __init__(self, rid, seed, **ranges):
        from mdpgen import request_header
        self.rid, self.seed, self.ranges = rid, seed, ranges
        self.S, self.A, self.k, self.gamma = request_header(rid, seed, **ranges)
        self.nnz, self.kmax = self.S * self.A * self.k, self.k

    def device_arrays(self):
        from mdpgen.cuda_gen import serving_request_cuda
        return serving_request_cuda(self.rid, self.seed, **self.ranges)[4:]


SERVE_MIX = dict(s_range=(1_000, 1_000_000), a_range=(2, 32), k_range=(4, 64), gammas=(0.9, 0.99, 0.999, 0.9999))


def run_serving(n, slots=4, seed=5):
    """Continuous-batching measurement on the serving stream: n requests with S
    log-uniform in [1e3, 1e6], A in [2, 32], k in [4, 64] entries per row and gamma in
    {0.9, 0.99, 0.999, 0.9999}, each drawn on the device at admission; Poisson
    arrivals at 0.8 of the one-at-a-time rate (and a burst of all n at once),
    admitted by a 120 GB HBM budget into `slots` concurrent solves, each solve one
    request or (batch_max 8) up to 8 requests through mdp_solve_batch."""
    import numpy as np

    from mdpgen.cuda_gen import load as load_gen
    from paper_2507_22538_gb300.serve import (Request, SolveService, fifo_one_at_a_time, latency_summary,
                                              solve_alone)
    load_gen()
    reqs = [Request(i, DeviceRequest(i, seed, **SERVE_MIX), tol=1e-8, alpha=1e-3) for i in range(n)]
    for r in reqs[:3]:
        solve_alone(r)  # warm-up
    alone = [solve_alone(r) for r in reqs]
    service = np.array([a.finished for a in alone])
    # the same solves stream-driven (the service and solve_alone run graph-driven solves)
    service_stream = np.array([solve_alone(r, graph=False).finished for r in reqs])
    rate = 0.8 / float(service.mean())
    gaps = np.random.default_rng(seed).exponential(1.0 / rate, size=n)
    arrivals = np.cumsum(gaps) - gaps[0]

    def drive(arr, batch_max, graph=True):
        svc = SolveService(slots=slots, hbm_budget=120 << 30, batch_max=batch_max, graph=graph).start()
        t0 = svc.now()
        for r, a in zip(reqs, arr):
            wait = t0 + a - svc.now()
            if wait > 0:
                time.sleep(wait)
            svc.submit(r)
        out = svc.wait(n)
        svc.close()
        summ = latency_summary(out)
        if batch_max > 1:
            summ.update(batch_max=batch_max, mean_batch=float(np.mean(svc.batches)), solves=len(svc.batches))
        summ["oom_retries"] = svc.oom_retries
        return out, summ, svc

    res, cont, svc = drive(arrivals, 1)
    # the same arrivals served by stream-driven solves
    _, cont_stream, _ = drive(arrivals, 1, graph=False)
    # the same arrivals, and a burst of all n at once, with waiting requests solved
    # together by mdp_solve_batch (up to 8 per call)
    resb, cont_b, _ = drive(arrivals, 8)
    burst = np.zeros(n)
    _, burst1, _ = drive(burst, 1)
    _, burst8, _ = drive(burst, 8)
    mism = []
    for tag, out in (("continuous", res), ("continuous_batched", resb)):
        for r in reqs:
            a, b = alone[r.rid], out[r.rid]
            if not (a.status == b.status and np.array_equal(a.V, b.V) and np.array_equal(a.pi, b.pi)):
                mism.append({"run": tag, "rid": r.rid, "status_alone": a.status, "status": b.status,
                             "error": b.error or a.error,
                             "outer": [a.outer_iters, b.outer_iters], "inner": [a.inner_iters, b.inner_iters],
                             "max_dV": float(np.max(np.abs(a.V - b.V))) if a.V.shape == b.V.shape and a.V.size else None})
    same = not mism
    nnz = np.array([r.data.nnz for r in reqs], dtype=np.float64)
    small = run_small_burst(slots=slots, seed=seed)
    return {"requests": n, "slots": slots, "hbm_budget_GB": 120, "arrival_rate_per_s": rate,
            "mix": "S log-uniform 1e3..1e6, A 2..32, k 4..64, gamma in {0.9,0.99,0.999,0.9999}, Dirichlet(1), "
                   "GMRES(30), alpha 1e-3, tol 1e-8; drawn on the device at admission (counted in the latency)",
            "entries_per_request": {"mean": float(nnz.mean()), "max": float(nnz.max())},
            "one_at_a_time_mean_s": float(service.mean()),
            "one_at_a_time_stream_driven_mean_s": float(service_stream.mean()),
            "continuous": cont, "one_at_a_time": fifo_one_at_a_time(arrivals, service),
            "one_at_a_time_stream_driven": fifo_one_at_a_time(arrivals, service_stream),
            "continuous_stream_driven": cont_stream,
            "continuous_batched": cont_b, "burst_continuous": burst1, "burst_batched": burst8,
            "peak_in_flight": svc.peak_in_flight, "results_equal_alone": bool(same),
            "statuses_alone": {int(k): int(v) for k, v in zip(*np.unique([a.status for a in alone], return_counts=True))},
            "mismatches": mism[:8], "n_mismatches": len(mism), "small_burst": small}


SMALL_MIX = dict(SERVE_MIX, s_range=(1_000, 4_096))


def run_small_burst(n=512, slots=4, seed=5, small_states=4096):
    """A burst of n small requests (the serving mix with S log-uniform in [1e3, 4096])
    arriving at once: one request per solve on the grid path, against the service
    gathering the pending small requests into mdp_solve_small_batch calls (one
    thread-block cluster per request).  A seeded sample is compared with the same
    request solved alone with the same routing."""
    import numpy as np

    from paper_2507_22538_gb300.serve import Request, SolveService, latency_summary, solve_alone
    reqs = [Request(i, DeviceRequest(i, seed + 1000, **SMALL_MIX), tol=1e-8, alpha=1e-3) for i in range(n)]
    out = {"requests": n, "mix": "the serving mix with S log-uniform in [1e3, 4096], all arriving at once"}
    for tag, ss in (("grid_one_per_solve", 0), ("cluster_batched", small_states)):
        for r in reqs[:3]:
            solve_alone(r, small_states=ss)  # warm-up
        svc = SolveService(slots=slots, hbm_budget=120 << 30, small_states=ss).start()
        for r in reqs:
            svc.submit(r)
        res = svc.wait(n)
        svc.close()
        summ = latency_summary(res)
        summ["mean_batch"] = float(np.mean(svc.batches))
        sample = np.random.default_rng(seed).choice(n, size=16, replace=False)
        summ["equal_alone"] = all(
            np.array_equal(solve_alone(reqs[i], small_states=ss).V, res[int(i)].V) for i in sample)
        summ["statuses"] = {int(k): int(v) for k, v in zip(*np.unique([x.status for x in res.values()],
                                                                       return_counts=True))}
        out[tag] = summ
    out["speedup_solves_per_s"] = out["cluster_batched"]["solves_per_s"] / out["grid_one_per_solve"]["solves_per_s"]
    return out


def run_serving_stream(n, slots=4, seed=5, calib=200, verify_frac=0.01, small_states=4096):
    """The full serving stream: n requests of the counter-based mix (S log-uniform in
    [1e3, 1e6], A in [2, 32], k in [4, 64], gamma in {0.9, 0.99, 0.999, 0.9999}, drawn
    on the device at admission) under Poisson arrivals at 0.8 of the one-at-a-time
    rate of plain FP64 solves measured on the first `calib` requests, admitted by a
    120 GB budget into `slots` concurrent solves; pending requests of at most
    small_states states are gathered into cluster-solver launches
    (mdp_solve_small_batch).  Results of the calibration requests and of a seeded
    sample of verify_frac of the rest are compared bit for bit with the same request
    solved alone with the same routing."""
    import numpy as np

    from mdpgen.cuda_gen import load as load_gen
    from paper_2507_22538_gb300.serve import Request, SolveService, latency_summary, solve_alone
    load_gen()
    reqs = [Request(i, DeviceRequest(i, seed, **SERVE_MIX), tol=1e-8, alpha=1e-3) for i in range(n)]
    for r in reqs[:3]:
        solve_alone(r)  # warm-up
    alone = {r.rid: solve_alone(r) for r in reqs[:calib]}
    service = np.array([a.finished for a in alone.values()])
    rate = 0.8 / float(service.mean())
    gaps = np.random.default_rng(seed).exponential(1.0 / rate, size=n)
    arrivals = np.cumsum(gaps) - gaps[0]
    rng = np.random.default_rng(seed + 1)
    sample = [int(i) for i in rng.choice(np.arange(calib, n), size=max(1, int(verify_frac * (n - calib))),
                                         replace=False)] if n > calib else []
    checked = set(alone) | set(sample)
    svc = SolveService(slots=slots, hbm_budget=120 << 30, keep=lambda rid: rid in checked,
                       small_states=small_states).start()
    t0 = svc.now()
    for r, a in zip(reqs, arrivals):
        wait = t0 + a - svc.now()
        if wait > 0:
            time.sleep(wait)
        svc.submit(r)
    out = svc.wait(n, timeout=4 * 3600)
    svc.close()
    summ = latency_summary(out)
    from paper_2507_22538_gb300.serve import is_small
    n_small = sum(is_small(r, small_states) for r in reqs)
    small_lat = [out[r.rid].latency for r in reqs if is_small(r, small_states)]
    for i in sample:
        alone[i] = solve_alone(reqs[i], small_states=small_states)
    for i in list(alone):
        if is_small(reqs[i], small_states):  # the calibration ran them on the grid path
            alone[i] = solve_alone(reqs[i], small_states=small_states)
    mism = [rid for rid, a in alone.items()
            if not (a.status == out[rid].status and np.array_equal(a.V, out[rid].V) and np.array_equal(a.pi, out[rid].pi))]
    statuses = {int(k): int(v) for k, v in zip(*np.unique([r.status for r in out.values()], return_counts=True))}
    nnz = np.array([r.data.nnz for r in reqs], dtype=np.float64)
    return {"requests": n, "slots": slots, "hbm_budget_GB": 120, "arrival_rate_per_s": rate,
            "mix": "S log-uniform 1e3..1e6, A 2..32, k 4..64, gamma in {0.9,0.99,0.999,0.9999}, Dirichlet(1), "
                   "GMRES(30), alpha 1e-3, tol 1e-8; drawn on the device at admission (counted in the latency)",
            "entries_per_request": {"mean": float(nnz.mean()), "max": float(nnz.max())},
            "calibration": {"requests": calib, "mean_solve_alone_s": float(service.mean())},
            "continuous": summ, "oom_retries": svc.oom_retries, "peak_in_flight": svc.peak_in_flight,
            "small_route": {"small_states": small_states, "requests": n_small,
                            "p50_s": float(np.percentile(small_lat, 50)) if small_lat else None,
                            "p99_s": float(np.percentile(small_lat, 99)) if small_lat else None,
                            "mean_batch_of_cluster_launches": float(np.mean([b for b in svc.batches if b > 1]))
                            if any(b > 1 for b in svc.batches) else 1.0},
            "statuses": statuses, "verified_alone": len(alone), "mismatches": mism[:8], "n_mismatches": len(mism)}


def sweep_variants(M, gamma, V, TV, pi, stream, sweeps=10):
    """The tuned launch shape of a handle's Bellman sweep, and the time per sweep of
    each rows-per-warp / value-load-width variant at the tuned tile (occupancy-limited
    grid); the tuned shape is restored afterwards."""
    import torch

    from paper_2507_22538_gb300 import mdp
    st, shape = mdp.mdp_get_sweep_shape(M.h)
    mdp.check(st, "mdp_get_sweep_shape")
    out = {"tuned": shape, "ms_per_sweep": {}}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for rpw, vb in ((32, 16), (32, 32), (64, 16), (64, 32)):
        mdp.check(mdp.mdp_set_sweep_shape(M.h, shape["tile_states"], rpw, vb, 0), "mdp_set_sweep_shape")
        for _ in range(2):
            mdp.check(mdp.mdp_bellman(M.h, gamma, V, TV, pi, None, stream), "mdp_bellman")
        e0.record(stream)
        for _ in range(sweeps):
            mdp.check(mdp.mdp_bellman(M.h, gamma, V, TV, pi, None, stream), "mdp_bellman")
        e1.record(stream)
        torch.cuda.synchronize()
        out["ms_per_sweep"][f"rows_per_warp={rpw},load_bytes={vb}"] = e0.elapsed_time(e1) / sweeps
    mdp.check(mdp.mdp_set_sweep_shape(M.h, shape["tile_states"], shape["rows_per_warp"], shape["value_load_bytes"],
                                      shape["blocks_per_sm"]), "mdp_set_sweep_shape")
    return out


MID_MIX = dict(SERVE_MIX, s_range=(65_537, 200_000))


def run_mid_batch(n=16, seed=7, reps=5):
    """n requests of the serving mix with S log-uniform in [65,537, 2e5] (above the
    cluster solver's limit), drawn on the device once: the solve calls alone (stream-
    and graph-driven, one request at a time) against mdp_solve_batch on all n (stream-
    driven: one host read per outer iteration and per GMRES cycle for the batch;
    graph-driven: the whole batch as one CUDA graph launch, built inside the call).
    Every mode gives every request the same V, policy and counts bit for bit."""
    import numpy as np
    import torch

    from mdpgen.cuda_gen import load as load_gen
    from paper_2507_22538_gb300 import mdp
    load_gen()
    stream = torch.cuda.current_stream()
    reqs = [DeviceRequest(i, seed, **MID_MIX) for i in range(n)]
    handles = []
    try:
        for r in reqs:
            rp, col, val, g = r.device_arrays()
            st, h = mdp.mdp_create(r.S, r.A, rp, col, val, g, True, stream)
            del rp, col, val, g
            mdp.check(st, "mdp_create")
            handles.append(h)
        V = [torch.zeros(r.S, dtype=torch.float64, device="cuda") for r in reqs]
        pi = [torch.empty(r.S, dtype=torch.int32, device="cuda") for r in reqs]

        def opts(graph):
            out = []
            for r in reqs:
                o = mdp.mdp_default_opts()
                o.gamma, o.atol_pi, o.alpha, o.gmres_restart, o.graph = r.gamma, 1e-8, 1e-3, 30, graph
                out.append(o)
            return out

        results, times = {}, {}
        for mode in ("alone_stream", "alone_graph", "batch_stream", "batch_graph"):
            graph = 1 if mode.endswith("graph") else 0
            ts = []
            for rep in range(reps + 1):  # rep 0 warms up (and builds the alone graphs)
                for v in V:
                    v.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                if mode.startswith("alone"):
                    stats, status = [], []
                    for i, o in enumerate(opts(graph)):
                        st, s1 = mdp.mdp_solve(handles[i], o, V[i], pi[i], stream)
                        status.append(st)
                        stats.append(s1)
                else:
                    st, status, stats = mdp.mdp_solve_batch(handles, opts(graph), V, pi, stream)
                    mdp.check(st, "mdp_solve_batch")
                torch.cuda.synchronize()
                ts.append(time.perf_counter() - t0)
            times[mode] = ts
            results[mode] = ([v.cpu().numpy() for v in V], [p.cpu().numpy() for p in pi], list(status),
                             [(x.outer_iters, int(x.inner_iters_total), x.final_residual) for x in stats])
        ref = results["alone_stream"]
        same = all(all(np.array_equal(a, b) for a, b in zip(results[m][0], ref[0])) and
                   all(np.array_equal(a, b) for a, b in zip(results[m][1], ref[1])) and
                   results[m][2] == ref[2] and results[m][3] == ref[3] for m in results)
        out = {"requests": n, "mix": "the serving mix with S log-uniform in [65537, 2e5], A 2..32, k 4..64, "
                                     "gamma in {0.9,0.99,0.999,0.9999}, GMRES(30), alpha 1e-3, tol 1e-8",
               "states": [r.S for r in reqs], "entries_total": int(sum(r.nnz for r in reqs)),
               "outer_inner": [list(x[:2]) for x in ref[3]], "statuses": [int(x) for x in ref[2]],
               "equal_bitwise_all_modes": bool(same),
               "timing": "host wall time of all n solves, median of %d after a warm-up" % reps}
        for m, ts in times.items():
            med = statistics.median(ts[1:])
            out[m] = {"s": med, "solves_per_s": n / med, "all_s": [round(t, 4) for t in ts]}
        out["alone_graph"]["first_call_s"] = times["alone_graph"][0]  # includes building every handle's graph
        out["batch_graph"]["first_call_s"] = times["batch_graph"][0]
        out["speedup_batch_graph_vs_alone_stream"] = out["alone_stream"]["s"] / out["batch_graph"]["s"]
        out["speedup_batch_graph_vs_batch_stream"] = out["batch_stream"]["s"] / out["batch_graph"]["s"]
        return out
    finally:
        for h in handles:
            mdp.mdp_destroy(h)


def run_small(steps=20):
    """The small random workload (S = 1000, A = 4, 8 entries per row, Dirichlet(1),
    gamma = 0.9, GMRES(30), alpha = 1e-3, tol = 1e-10): time to solution of the
    stream-driven mdp_solve against the graph-driven one (opts.graph: the whole of
    Algorithm 1 in one CUDA graph launch), and the first graph call, which builds
    and instantiates the graph.  Each time is the wall time of one blocking call."""
    import torch

    from mdpgen import random_sparse
    from paper_2507_22538_gb300 import mdp
    m = random_sparse(1000, 4, 8, 0.9, seed=1)
    stream = torch.cuda.current_stream()
    out = {"workload": "random sparse S=1000, A=4, k=8, Dirichlet(1), gamma=0.9, GMRES(30), alpha=1e-3, tol=1e-10",
           "timing": "host wall time of each blocking mdp_solve call, median of %d" % steps}
    with mdp.MDP.from_data(m, stream) as M:
        V = torch.zeros(m.S, dtype=torch.float64, device="cuda")
        pi = torch.empty(m.S, dtype=torch.int32, device="cuda")
        o = mdp.mdp_default_opts()
        o.gamma, o.atol_pi, o.alpha, o.gmres_restart = m.gamma, 1e-10, 1e-3, 30
        for name, graph in (("stream", 0), ("graph", 1)):
            o.graph = graph
            times = []
            for i in range(steps + 3):
                V.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st, stats = mdp.mdp_solve(M.h, o, V, pi, stream)
                times.append(time.perf_counter() - t0)
                mdp.check(st, "mdp_solve")
            out[name] = {"ms": statistics.median(times[3:]) * 1e3, "first_call_ms": times[0] * 1e3,
                         "outer": stats.outer_iters, "inner": stats.inner_iters_total,
                         "launches": stats.kernel_launches, "final_residual": stats.final_residual}
    out["speedup_graph"] = out["stream"]["ms"] / out["graph"]["ms"]
    # the same problem solved inside one thread-block cluster (mdp_solve_small_batch, n = 1),
    # and a batch of 256 such problems (seeds 1..256) in one call
    with mdp.MDP.from_data(m, stream) as M:
        V = torch.zeros(m.S, dtype=torch.float64, device="cuda")
        pi = torch.empty(m.S, dtype=torch.int32, device="cuda")
        o = mdp.mdp_default_opts()
        o.gamma, o.atol_pi, o.alpha, o.gmres_restart = m.gamma, 1e-10, 1e-3, 30
        times = []
        for i in range(steps + 3):
            V.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, status, stats = mdp.mdp_solve_small_batch([M.h], [o], [V], [pi], stream)
            times.append(time.perf_counter() - t0)
            mdp.check(st, "mdp_solve_small_batch")
            mdp.check(status[0], "small batch member")
        out["cluster"] = {"ms": statistics.median(times[3:]) * 1e3, "outer": stats[0].outer_iters,
                          "inner": stats[0].inner_iters_total, "launches": stats[0].kernel_launches,
                          "final_residual": stats[0].final_residual}
    out["speedup_cluster_vs_graph"] = out["graph"]["ms"] / out["cluster"]["ms"]
    nb = 256
    ms_b = [random_sparse(1000, 4, 8, 0.9, seed=i + 1) for i in range(nb)]
    Ms = [mdp.MDP.from_data(x, stream) for x in ms_b]
    try:
        Vs = [torch.zeros(x.S, dtype=torch.float64, device="cuda") for x in ms_b]
        ps = [torch.empty(x.S, dtype=torch.int32, device="cuda") for x in ms_b]
        opts = []
        for x in ms_b:
            o = mdp.mdp_default_opts()
            o.gamma, o.atol_pi, o.alpha, o.gmres_restart = x.gamma, 1e-10, 1e-3, 30
            opts.append(o)
        times = []
        for i in range(4):
            for v in Vs:
                v.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st, status, stats = mdp.mdp_solve_small_batch([M.h for M in Ms], opts, Vs, ps, stream)
            times.append(time.perf_counter() - t0)
            mdp.check(st, "mdp_solve_small_batch")
            assert all(x == mdp.MDP_OK for x in status), status
        tb = statistics.median(times[1:])
        out["cluster_batch"] = {"problems": nb, "s": tb, "solves_per_s": nb / tb,
                                "one_at_a_time_graph_solves_per_s": 1e3 / out["graph"]["ms"],
                                "what": "256 random MDPs of the same shape (seeds 1..256) in one "
                                        "mdp_solve_small_batch call, each on one 2-block cluster"}
    finally:
        for M in Ms:
            M.close()
    return out


def run_stress(sweeps=10):
    """The bandwidth-stress random workload at full size (S = 2e6, A = 32, 32 entries
    per row = 2.05e9 entries, Dirichlet(0.5) quantised to 2^-11, gamma = 0.99), built on
    the device: event-timed Bellman sweeps against the HBM roofline, and one FP64 and
    one mixed-precision solve (GMRES(30), alpha = 1e-4, tol = 1e-8)."""
    import torch

    from mdpgen.torch_gen import random_sparse_device
    from paper_2507_22538_gb300 import mdp
    Sx, Ax, Kx, gx = 2_000_000, 32, 32, 0.99
    t0 = time.perf_counter()
    rp, col, val, g = random_sparse_device(Sx, Ax, Kx, gx, 21, conc=0.5, quant_bits=11)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    out = {"workload": "random sparse S=2e6, A=32, k=32 (2.05e9 entries), Dirichlet(0.5) quantised to 2^-11, "
                       "gamma=0.99, built on the device", "generate_s": t_gen}
    with mdp.MDP(Sx, Ax, rp, col, val, g, stream) as M:
        del rp, col, val, g
        torch.cuda.empty_cache()
        st_t, tile_states, _ = mdp.mdp_tune(M.h, gx, stream)
        mdp.check(st_t, "mdp_tune")
        out["tile_states"] = tile_states
        V = torch.zeros(Sx, dtype=torch.float64, device="cuda")
        TV = torch.empty_like(V)
        pi = torch.empty(Sx, dtype=torch.int32, device="cuda")
        out["sweep_shape"] = sweep_variants(M, gx, V, TV, pi, stream, sweeps=4)
        for _ in range(3):
            mdp.check(mdp.mdp_bellman(M.h, gx, V, TV, pi, None, stream), "mdp_bellman")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(sweeps):
            mdp.check(mdp.mdp_bellman(M.h, gx, V, TV, pi, None, stream), "mdp_bellman")
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / sweeps
        R = Sx * Ax
        nbytes = R * Kx * 12 + R * 16 + Sx * 20
        peak, _ = load_peaks()
        out["bellman"] = {"ms_per_sweep": ms, "bytes": nbytes, "GB/s": nbytes / ms / 1e6,
                          "frac": nbytes / ms / 1e6 / peak, "fp64_fma_per_s": R * Kx / (ms * 1e-3)}
        # the certified low-precision sweep at the workload's stated precision (binary16 values,
        # int32 columns): same outputs bit for bit
        for _ in range(3):
            mdp.check(mdp.mdp_bellman_lowp(M.h, gx, V, TV, pi, None, stream), "mdp_bellman_lowp")
        e0.record(stream)
        for _ in range(sweeps):
            mdp.check(mdp.mdp_bellman_lowp(M.h, gx, V, TV, pi, None, stream), "mdp_bellman_lowp")
        e1.record(stream)
        torch.cuda.synchronize()
        ms_l = e0.elapsed_time(e1) / sweeps
        lb = lowp_bytes(Sx, Ax, Kx)
        out["bellman_lowp"] = {"ms_per_sweep": ms_l, "bytes": lb, "GB/s": lb / ms_l / 1e6, "frac": lb / ms_l / 1e6 / peak,
                               "l2_sectors_per_sweep": R * Kx, "gather_sector_GBps": R * Kx * 32 / ms_l / 1e6,
                               "what": "binary16 values + int32 columns (the workload's stated storage); each "
                                       "random V gather is its own 32-byte L2 sector"}
        ref = None
        for name, prec, lp in (("solve_f64", mdp.MDP_PREC_F64, 0), ("solve_mixed", mdp.MDP_PREC_MIXED, 0),
                               ("solve_mixed_lowp_sweep", mdp.MDP_PREC_MIXED, 1)):
            o = mdp.mdp_default_opts()
            o.gamma, o.atol_pi, o.alpha, o.gmres_restart, o.precision = gx, 1e-8, 1e-4, 30, prec
            o.lowp_sweep = lp
            for rep in range(2):  # the first call allocates the Krylov workspace
                V.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st, stats = mdp.mdp_solve(M.h, o, V, pi, stream)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
            mdp.check(st, "mdp_solve")
            out[name] = {"s": dt, "outer": stats.outer_iters, "inner": stats.inner_iters_total,
                         "final_residual": stats.final_residual, "policy_value_bytes": stats.policy_value_bytes,
                         "sweep_value_bytes": stats.bellman_value_bytes}
            Vh, pih = V.cpu().numpy(), pi.cpu().numpy()
            # costs lie in [0, 1): |g| < 1
            out[name]["error"] = error_statement(Vh, pih, stats.final_residual, gx, Kx, 1.0, ref)
            ref = ref or (Vh, pih)
    torch.cuda.empty_cache()
    return out


def run_pendulum():
    """The pendulum grid at full size (1000 x 1000 states, A = 9, 4 entries per row,
    gamma = 0.9999): Algorithm 1 to tol = 1e-8 with the Table 1 defaults (alpha = 1e-4,
    at most 1000 outer and 1000 inner iterations) and GMRES(30), FP64 and mixed, and
    with TFQMR; then the variant whose bilinear weights are rounded to 2^-8 (exact in
    bfloat16), FP64 against mixed with bfloat16 policy values."""
    import numpy as np
    import torch

    from mdpgen import pendulum_grid
    from paper_2507_22538_gb300 import mdp
    out = {"workload": "pendulum grid 1000 x 1000, A=9, k=4, gamma=0.9999, Ts=0.01", "tol": 1e-8, "alpha": 1e-4}
    stream = torch.cuda.current_stream()
    for tag, qb in (("", None), ("bf16_exact_", 8)):
        m = pendulum_grid(1000, 1000, 9, 0.9999, seed=3, quant_bits=qb)
        runs = (("gmres_f64", mdp.MDP_GMRES, mdp.MDP_PREC_F64), ("gmres_mixed", mdp.MDP_GMRES, mdp.MDP_PREC_MIXED))
        if qb is None:
            runs += (("tfqmr_f64", mdp.MDP_TFQMR, mdp.MDP_PREC_F64),)
        with mdp.MDP.from_data(m, stream) as M:
            V = torch.zeros(m.S, dtype=torch.float64, device="cuda")
            pi = torch.empty(m.S, dtype=torch.int32, device="cuda")
            ref = None
            gnorm = float(np.max(np.abs(m.g)))
            for name, inner, prec in runs:
                o = mdp.mdp_default_opts()
                o.gamma, o.atol_pi, o.alpha, o.gmres_restart, o.inner, o.precision = 0.9999, 1e-8, 1e-4, 30, inner, prec
                V.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st, stats = mdp.mdp_solve(M.h, o, V, pi, stream)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                out[tag + name] = {"s": dt, "status": st, "outer": stats.outer_iters, "inner": stats.inner_iters_total,
                                   "final_residual": stats.final_residual,
                                   "policy_value_bytes": stats.policy_value_bytes}
                Vh, pih = V.cpu().numpy(), pi.cpu().numpy()
                out[tag + name]["error"] = error_statement(Vh, pih, stats.final_residual, 0.9999, 4, gnorm, ref)
                ref = ref or (Vh, pih)
    return out


def run_bellman_only(args):
    """Time mdp_bellman alone on the banded workload, or (--workload random) on the
    bandwidth-stress random workload's generator (A = 32, 32 entries per row,
    Dirichlet(0.5) quantised to 2^-11, built on the device), at any size; one JSON line."""
    import torch

    from mdpgen import MDPData, banded_birth_death, random_value_vector
    from paper_2507_22538_gb300 import mdp
    from paper_2507_22538_gb300.build import build
    build()
    if args.workload == "random":
        from mdpgen.torch_gen import random_sparse_device
        return run_bellman_only_random(args, random_sparse_device, random_value_vector)
    m = banded_birth_death(args.states, A, H, GAMMA, quant_bits=args.quant_bits or None)
    stream = torch.cuda.current_stream()
    with mdp.MDP.from_data(m, stream) as M:
        st_t, tile_states, _ = mdp.mdp_tune(M.h, GAMMA, stream)
        mdp.check(st_t, "mdp_tune")
        V = torch.from_numpy(random_value_vector(m.S, 1, 1000.0)).cuda()
        TV = torch.empty_like(V)
        pi = torch.empty(m.S, dtype=torch.int32, device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms_lowp = None
        if args.quant_bits:  # the certified low-precision sweep on the binary16-exact variant
            for _ in range(2):
                mdp.check(mdp.mdp_bellman_lowp(M.h, GAMMA, V, TV, pi, None, stream), "mdp_bellman_lowp")
            e0.record(stream)
            for _ in range(args.bellman_only):
                mdp.check(mdp.mdp_bellman_lowp(M.h, GAMMA, V, TV, pi, None, stream), "mdp_bellman_lowp")
            e1.record(stream)
            torch.cuda.synchronize()
            ms_lowp = e0.elapsed_time(e1) / args.bellman_only
        for _ in range(2):
            mdp.check(mdp.mdp_bellman(M.h, GAMMA, V, TV, pi, None, stream), "mdp_bellman")
        e0.record(stream)
        for _ in range(args.bellman_only):
            mdp.check(mdp.mdp_bellman(M.h, GAMMA, V, TV, pi, None, stream), "mdp_bellman")
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.bellman_only
        # the greedy policy's rows gathered (Algorithm 1 step 4) and applied once: mdp_policy_apply
        Y = torch.empty_like(V)
        mdp.check(mdp.mdp_policy_apply(M.h, GAMMA, pi, V, Y, stream), "mdp_policy_apply")
        e0.record(stream)
        for _ in range(args.bellman_only):
            mdp.check(mdp.mdp_policy_apply(M.h, GAMMA, pi, V, Y, stream), "mdp_policy_apply")
        e1.record(stream)
        torch.cuda.synchronize()
        ms_pa = e0.elapsed_time(e1) / args.bellman_only
    R = m.S * A
    nbytes = R * K_ROW * 12 + (R + 1) * 8 + R * 8 + m.S * 8 + m.S * 12
    # gather: read pi and the S chosen rows (12 B per entry) and g; write the rows and g_pi
    gather_bytes = m.S * (4 + 8 + 8) + 2 * m.S * K_ROW * 12
    peak, _ = load_peaks()
    out = {"mode": "bellman_only", "S": m.S, "ms_per_sweep": ms, "bytes": nbytes,
           "GB/s": nbytes / ms / 1e6, "frac": nbytes / ms / 1e6 / peak,
           "ms_per_gather_and_apply": ms_pa, "gather_bytes": gather_bytes, "tile_states": tile_states}
    if ms_lowp:
        lb = lowp_bytes(m.S, A, K_ROW)
        out["lowp"] = {"ms_per_sweep": ms_lowp, "bytes": lb, "GB/s": lb / ms_lowp / 1e6,
                       "frac": lb / ms_lowp / 1e6 / peak}
    print(json.dumps(out), flush=True)
    return 0


def run_bellman_only_random(args, random_sparse_device, random_value_vector):
    import torch

    from paper_2507_22538_gb300 import mdp
    Sx, Ax, Kx, gx = args.states, 32, 32, 0.99
    rp, col, val, g = random_sparse_device(Sx, Ax, Kx, gx, 21, conc=0.5, quant_bits=11)
    stream = torch.cuda.current_stream()
    with mdp.MDP(Sx, Ax, rp, col, val, g, stream) as M:
        del rp, col, val, g
        torch.cuda.empty_cache()
        st_t, tile_states, _ = mdp.mdp_tune(M.h, gx, stream)
        mdp.check(st_t, "mdp_tune")
        V = torch.from_numpy(random_value_vector(Sx, 1, 100.0)).cuda()
        TV = torch.empty_like(V)
        pi = torch.empty(Sx, dtype=torch.int32, device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        times = {}
        for name, fn in (("f64", mdp.mdp_bellman), ("lowp", mdp.mdp_bellman_lowp)):
            for _ in range(2):
                mdp.check(fn(M.h, gx, V, TV, pi, None, stream), name)
            e0.record(stream)
            for _ in range(args.bellman_only):
                mdp.check(fn(M.h, gx, V, TV, pi, None, stream), name)
            e1.record(stream)
            torch.cuda.synchronize()
            times[name] = e0.elapsed_time(e1) / args.bellman_only
        ms = times["f64"]
    R = Sx * Ax
    nbytes = R * Kx * 12 + R * 16 + Sx * 20
    lb = lowp_bytes(Sx, Ax, Kx)
    peak, _ = load_peaks()
    print(json.dumps({"mode": "bellman_only", "workload": "random", "S": Sx, "A": Ax, "k": Kx, "ms_per_sweep": ms,
                      "bytes": nbytes, "GB/s": nbytes / ms / 1e6, "frac": nbytes / ms / 1e6 / peak,
                      "gathers_per_s": R * Kx / (ms * 1e-3), "tile_states": tile_states,
                      "lowp": {"ms_per_sweep": times["lowp"], "bytes": lb, "GB/s": lb / times["lowp"] / 1e6,
                               "frac": lb / times["lowp"] / 1e6 / peak}}), flush=True)
    return 0


def run_solve_only(args):
    """Time W + K solves of the workload at one precision, one JSON line (profiling
    aid: the launch list of a single solve without the rest of the bench)."""
    import torch

    from mdpgen import banded_birth_death
    from paper_2507_22538_gb300 import mdp
    from paper_2507_22538_gb300.build import build
    build()
    m = banded_birth_death(args.states, A, H, GAMMA, quant_bits=args.quant_bits or None)
    stream = torch.cuda.current_stream()
    prec = mdp.MDP_PREC_MIXED if args.solve_only == "mixed" else mdp.MDP_PREC_F64
    with mdp.MDP.from_data(m, stream) as M:
        mdp.check(mdp.mdp_tune(M.h, GAMMA, stream)[0], "mdp_tune")
        V = torch.zeros(m.S, dtype=torch.float64, device="cuda")
        pi = torch.empty(m.S, dtype=torch.int32, device="cuda")
        o = mdp.mdp_default_opts()
        o.gamma, o.atol_pi, o.alpha, o.gmres_restart, o.inner, o.precision = GAMMA, TOL, ALPHA, RESTART, mdp.MDP_GMRES, prec
        o.lowp_sweep = 1 if args.quant_bits else 0  # the binary16-exact variant runs the certified binary16 sweep
        o.record_timing = 1 if args.timing else 0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        launches = 0
        for i in range(args.warmup + args.steps):
            if i == args.warmup:
                torch.cuda.synchronize()
                e0.record(stream)
            V.zero_()
            st, stats = mdp.mdp_solve(M.h, o, V, pi, stream)
            mdp.check(st, "mdp_solve")
            launches = stats.kernel_launches
        e1.record(stream)
        torch.cuda.synchronize()
    out = {"mode": "solve_only", "precision": args.solve_only, "S": m.S,
           "ms_per_solve": e0.elapsed_time(e1) / max(1, args.steps), "launches_per_solve": launches,
           "outer": stats.outer_iters, "inner": stats.inner_iters_total}
    if args.timing:  # the last solve's event-timed kernels (record_timing)
        out.update(bellman_ms=stats.bellman_ms / max(1, stats.bellman_sweeps),
                   matvec_ms=stats.matvec_ms / max(1, stats.matvecs_timed),
                   gs_pair_ms=stats.gs_ms / max(1, stats.gs_timed),
                   gs_tflops=stats.gs_flops / (stats.gs_ms * 1e-3) / 1e12 if stats.gs_ms > 0 else None)
    print(json.dumps(out), flush=True)
    return 0


def run_inner_only(args):
    """Time a fixed number of GMRES(30) iterations of mdp_policy_eval on the policy
    'always action 0' of the banded workload, built as a one-action MDP (0.4 GB)."""
    import numpy as np
    import torch

    from mdpgen import MDPData, banded_birth_death
    from paper_2507_22538_gb300 import mdp
    from paper_2507_22538_gb300.build import build
    build()
    full = banded_birth_death(args.states, A, H, GAMMA)
    rows = np.arange(args.states, dtype=np.int64) * A  # row (s, 0)
    k = K_ROW
    col = full.col.reshape(-1, k)[rows].ravel()
    val = full.val.reshape(-1, k)[rows].ravel()
    m = MDPData(args.states, 1, np.arange(args.states + 1, dtype=np.int64) * k, col, val, full.g[rows], GAMMA)
    del full
    stream = torch.cuda.current_stream()
    with mdp.MDP.from_data(m, stream) as M:
        pi = torch.zeros(m.S, dtype=torch.int32, device="cuda")
        v0 = torch.zeros(m.S, dtype=torch.float64, device="cuda")
        v = torch.empty_like(v0)
        mdp.mdp_policy_eval(M.h, GAMMA, pi, v0, v, mdp.MDP_GMRES, RESTART, 1.0, 0.0, 30, stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, it, res = mdp.mdp_policy_eval(M.h, GAMMA, pi, v0, v, mdp.MDP_GMRES, RESTART, 1.0, 0.0, args.inner_only,
                                          stream)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    print(json.dumps({"mode": "inner_only", "S": m.S, "iterations": it, "ms_per_iteration": dt * 1e3 / max(it, 1),
                      "residual": res}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--reference-states", type=int, default=0, metavar="S",
                    help="test aid for --impl reference: solve the workload's generator at S states instead of "
                         "1e6 (the line's config names the size)")
    ap.add_argument("--cpu-oracle-worker", default=None, metavar="NPZ",
                    help=argparse.SUPPRESS)  # child process: one timed oracle solve, V and pi saved to NPZ
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-quantized", dest="quantized", action="store_false",
                    help="skip the binary16-exact variant of the workload")
    ap.add_argument("--no-pendulum", dest="pendulum", action="store_false",
                    help="skip the full-size pendulum grid solves (gamma = 0.9999)")
    ap.add_argument("--no-stress", dest="stress", action="store_false",
                    help="skip the 2.05e9-entry random workload (sweep roofline and two solves)")
    ap.add_argument("--serve", type=int, default=200, metavar="N",
                    help="requests of the continuous-batching measurement added to the line (0: skip)")
    ap.add_argument("--bellman-only", type=int, default=0, metavar="SWEEPS",
                    help="profiling aid: time SWEEPS mdp_bellman calls on the workload (no bench line)")
    ap.add_argument("--workload", choices=["banded", "random"], default="banded",
                    help="with --bellman-only: the banded workload, or the random bandwidth-stress generator "
                         "(A = 32, k = 32) at --states states")
    ap.add_argument("--quant-bits", type=int, default=0,
                    help="with --bellman-only or --solve-only on the banded workload: round the band to multiples of "
                         "2^-this (11: exact in binary16) and also time (bellman-only) or use (solve-only) the "
                         "certified low-precision sweep")
    ap.add_argument("--states", type=int, default=S, help="with --bellman-only/--inner-only/--solve-only: number of states")
    ap.add_argument("--inner-only", type=int, default=0, metavar="ITERS",
                    help="profiling aid: ITERS GMRES(30) iterations of mdp_policy_eval on the rows of action 0 "
                         "of the workload (a one-action MDP; no bench line)")
    ap.add_argument("--solve-only", choices=["f64", "mixed"], default=None,
                    help="profiling aid: W + K solves of the workload at this precision (no bench line)")
    ap.add_argument("--timing", action="store_true",
                    help="with --solve-only: record_timing on, and the event-timed kernel averages in the line")
    ap.add_argument("--serve-stream", type=int, default=0, metavar="N",
                    help="only the full serving stream of N requests (no bench line)")
    ap.add_argument("--stream", type=int, default=10000, metavar="N",
                    help="requests of the full serving stream added to the line (0: skip)")
    ap.add_argument("--small-only", action="store_true",
                    help="only the small-workload stream vs graph measurement (no bench line)")
    ap.add_argument("--mid-batch-only", action="store_true",
                    help="only the mid-size batch measurement, alone vs batched, stream vs graph (no bench line)")
    args = ap.parse_args()
    if args.cpu_oracle_worker:
        return run_cpu_oracle_worker(args)
    if args.serve_stream:
        import torch
        from paper_2507_22538_gb300.build import build
        build()
        print(json.dumps({"mode": "serve_stream", **run_serving_stream(args.serve_stream)}), flush=True)
        return 0
    if args.small_only:
        import torch
        from paper_2507_22538_gb300.build import build
        build()
        print(json.dumps({"mode": "small_only", **run_small()}), flush=True)
        return 0
    if args.mid_batch_only:
        import torch
        from paper_2507_22538_gb300.build import build
        build()
        print(json.dumps({"mode": "mid_batch_only", **run_mid_batch()}), flush=True)
        return 0
    if args.solve_only:
        return run_solve_only(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.bellman_only:
        return run_bellman_only(args)
    if args.inner_only:
        return run_inner_only(args)

    world, rank, local = dist_env()
    oracle_child, oracle_npz = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the FP64 oracle on the same workload, timed on one host core in a child process
        # started before any GPU call, while the GPU measurements below proceed
        fd, oracle_npz = tempfile.mkstemp(suffix=".npz")
        os.close(fd)
        oracle_child = subprocess.Popen([sys.executable, os.path.abspath(__file__), "--cpu-oracle-worker",
                                         oracle_npz], stdin=subprocess.PIPE, stdout=subprocess.PIPE,
                                        stderr=subprocess.PIPE, text=True)

    t_main = time.perf_counter()
    import numpy as np
    import torch

    from mdpgen import banded_birth_death
    from paper_2507_22538_gb300 import mdp

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2507_22538_gb300.build import build
    if rank == 0 or world == 1:
        build()
    if dist:
        dist.barrier()
    mdp.load()

    m = banded_birth_death(S, A, H, GAMMA)
    stream = torch.cuda.current_stream()
    M = mdp.MDP.from_data(m, stream)
    st_t, tile_states, tune_ms = mdp.mdp_tune(M.h, GAMMA, stream)  # launch-shape autotuner, outside the timing
    mdp.check(st_t, "mdp_tune")
    V = torch.zeros(S, dtype=torch.float64, device="cuda")
    pi = torch.empty(S, dtype=torch.int32, device="cuda")
    shape_info = sweep_variants(M, GAMMA, V, torch.empty_like(V), pi, stream)
    opts = mdp.mdp_default_opts()
    opts.gamma, opts.atol_pi, opts.alpha, opts.gmres_restart = GAMMA, TOL, ALPHA, RESTART
    opts.inner, opts.record_timing = mdp.MDP_GMRES, 1

    def step(o=opts):
        V.zero_()
        st, stats = mdp.mdp_solve(M.h, o, V, pi, stream)
        mdp.check(st, "mdp_solve")
        return stats.as_dict()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    totals = {}
    with ClockSampler(local) as clk:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        marks = []
        for _ in range(args.steps):
            s = step()
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(stream)
            marks.append(ev)
            for key in ("outer_iters", "inner_iters_total", "kernel_launches", "bellman_sweeps", "bellman_ms",
                        "inner_ms", "inner_bytes", "matvec_ms", "matvecs_timed", "matvec_bytes", "matvec_flops", "gs_ms",
                        "gs_flops", "gs_timed"):
                totals[key] = totals.get(key, 0) + s[key]
            totals["final_residual"] = max(totals.get("final_residual", 0.0), s["final_residual"])
        e1.record(stream)
        torch.cuda.synchronize()
        step_ms = [e0.elapsed_time(marks[0])] + [a.elapsed_time(b) for a, b in zip(marks, marks[1:])]
    if dist:
        dist.barrier()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, "cuda")
    clocks = clk.summary()
    V64, pi64 = V.cpu().numpy().copy(), pi.cpu().numpy().copy()
    s64_res = s["final_residual"]
    gnorm = float(np.max(np.abs(m.g)))

    # the same solves without per-sweep event timing, stream-driven and as one CUDA graph each
    graph_cmp = {}
    for name, graph in (("stream", 0), ("graph", 1)):
        gopts = mdp.mdp_default_opts()
        for f, _ in mdp.mdp_solve_opts._fields_:
            setattr(gopts, f, getattr(opts, f))
        gopts.record_timing, gopts.graph = 0, graph
        for _ in range(max(1, args.warmup)):
            step(gopts)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            s = step(gopts)
        e1.record(stream)
        torch.cuda.synchronize()
        graph_cmp[name + "_ms"] = e0.elapsed_time(e1) / args.steps
        graph_cmp[name + "_outer_inner"] = [s["outer_iters"], s["inner_iters_total"]]
    graph_cmp["what"] = ("the timed solves without per-sweep event timing: stream-driven, and as one CUDA graph "
                         "launch per solve (opts.graph)")

    # the same solves with the mixed-precision inner solver (FP32 Arnoldi, FP64 refinement)
    mopts = mdp.mdp_default_opts()
    for f, _ in mdp.mdp_solve_opts._fields_:
        setattr(mopts, f, getattr(opts, f))
    mopts.precision = mdp.MDP_PREC_MIXED
    for _ in range(args.warmup):
        step(mopts)
    torch.cuda.synchronize()
    mtot = {}
    e0.record(stream)
    for _ in range(args.steps):
        s = step(mopts)
        for key in ("outer_iters", "inner_iters_total", "kernel_launches", "inner_ms", "inner_bytes"):
            mtot[key] = mtot.get(key, 0) + s[key]
        mtot["final_residual"] = max(mtot.get("final_residual", 0.0), s["final_residual"])
    e1.record(stream)
    torch.cuda.synchronize()
    mixed_ms = e0.elapsed_time(e1) / args.steps
    Vmx, pimx = V.cpu().numpy().copy(), pi.cpu().numpy().copy()
    mixed_res = s["final_residual"]

    # the quantised variant of the workload (binomial band rounded to multiples of 2^-11 so
    # that every probability is exact in binary16): FP64 path vs mixed path with binary16
    # policy rows, both on the same quantised MDP
    quant = None
    if args.quantized:
        M.close()
        mq = banded_birth_death(S, A, H, GAMMA, quant_bits=11)
        Mq = mdp.MDP.from_data(mq, stream)

        def qstep(o):
            V.zero_()
            st, stats = mdp.mdp_solve(Mq.h, o, V, pi, stream)
            mdp.check(st, "mdp_solve")
            return stats.as_dict()

        quant = {}
        qref = None
        lopts, lmopts = mdp.mdp_default_opts(), mdp.mdp_default_opts()
        for f, _ in mdp.mdp_solve_opts._fields_:
            setattr(lopts, f, getattr(opts, f))
            setattr(lmopts, f, getattr(mopts, f))
        lopts.lowp_sweep = lmopts.lowp_sweep = 1  # the certified binary16 sweep (same results bit for bit)
        for name, o in (("f64", opts), ("mixed", mopts), ("f64_lowp_sweep", lopts), ("mixed_lowp_sweep", lmopts)):
            for _ in range(args.warmup):
                qstep(o)
            torch.cuda.synchronize()
            e0.record(stream)
            its = []
            sw_ms, sw_n, rows64 = 0.0, 0, 0
            for _ in range(args.steps):
                s = qstep(o)
                its.append((s["outer_iters"], s["inner_iters_total"], s["policy_value_bytes"], s["final_residual"]))
                sw_ms += s["bellman_ms"]
                sw_n += s["bellman_sweeps"]
                rows64 += s["bellman_rows_fp64"]
            e1.record(stream)
            torch.cuda.synchronize()
            quant[name] = {"ms_per_step": e0.elapsed_time(e1) / args.steps, "outer": its[-1][0],
                           "inner": its[-1][1], "policy_value_bytes": its[-1][2],
                           "sweep_value_bytes": s["bellman_value_bytes"], "sweep_ms": sw_ms / max(1, sw_n),
                           "max_final_residual": max(i[3] for i in its)}
            if o.lowp_sweep:
                lb = lowp_bytes(S, A, K_ROW)
                quant[name]["sweep_GBps"] = lb / (quant[name]["sweep_ms"] * 1e-3) / 1e9
                quant[name]["sweep_frac"] = quant[name]["sweep_GBps"] / load_peaks()[0]
                quant[name]["rows_fp64_per_state_and_sweep"] = rows64 / max(1, sw_n) / S
            Vq, piq = V.cpu().numpy().copy(), pi.cpu().numpy().copy()
            quant[name]["error"] = error_statement(Vq, piq, its[-1][3], GAMMA, K_ROW, float(np.max(np.abs(mq.g))),
                                                   qref)
            qref = qref or (Vq, piq)
        quant["speedup_mixed_vs_f64"] = quant["f64"]["ms_per_step"] / quant["mixed"]["ms_per_step"]
        quant["speedup_mixed_lowp_sweep_vs_f64"] = (quant["f64"]["ms_per_step"] /
                                                    quant["mixed_lowp_sweep"]["ms_per_step"])
        quant["lowp_sweep_bit_identical"] = all(
            quant[a]["error"].get("max_abs_diff_vs_fp64_gpu", 0.0) == 0.0 for a in ("f64_lowp_sweep",))
        Mq.close()
        # end to end from pinned host buffers with the values in binary16 (exact for this MDP)
        # against the same values in binary64: create + mixed solve + read back
        qe = {}
        for tag, vals in (("binary16_values", torch.from_numpy(mq.val).to(torch.float16)),
                          ("binary64_values", torch.from_numpy(mq.val))):
            host = [torch.from_numpy(mq.row_ptr).pin_memory(), torch.from_numpy(mq.col).pin_memory(),
                    vals.pin_memory(), torch.from_numpy(mq.g).pin_memory()]
            times = []
            for i in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st, hq = mdp.mdp_create(S, A, *host, False, stream)
                mdp.check(st, "mdp_create")
                V.zero_()
                st, _ = mdp.mdp_solve(hq, lmopts, V, pi, stream)
                mdp.check(st, "mdp_solve")
                Vh_q = V.to("cpu", non_blocking=True)
                pih_q = pi.to("cpu", non_blocking=True)
                torch.cuda.synchronize()
                mdp.mdp_destroy(hq)
                if i:
                    times.append(time.perf_counter() - t0)
            if times:
                qe[tag] = {"s": sum(times) / len(times),
                           "h2d_bytes": int(sum(t.numel() * t.element_size() for t in host))}
            del host
        quant["e2e_mixed_solve"] = qe
        quant["what"] = ("banded workload with the band's probabilities rounded to multiples of 2^-11 "
                         "(exact in binary16); the mixed path reads binary16 policy rows")
        del mq
        M = None

    # end to end through the C ABI from pinned host buffers: upload + layout + solve + read back
    pinned = {k: torch.from_numpy(getattr(m, k)).pin_memory() for k in ("row_ptr", "col", "val", "g")}
    h2d = sum(int(t.numel() * t.element_size()) for t in pinned.values())
    Vh = torch.empty(S, dtype=torch.float64).pin_memory()
    pih = torch.empty(S, dtype=torch.int32).pin_memory()
    d2h = S * 8 + S * 4
    if M is not None:
        M.close()
    torch.cuda.synchronize()
    # the call a user makes: the graph-driven solve, without per-sweep event timing
    eopts = mdp.mdp_default_opts()
    for f, _ in mdp.mdp_solve_opts._fields_:
        setattr(eopts, f, getattr(opts, f))
    eopts.record_timing, eopts.graph = 0, 1
    e2e_times = []
    for i in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
        t0 = time.perf_counter()
        st, h = mdp.mdp_create(S, A, pinned["row_ptr"], pinned["col"], pinned["val"], pinned["g"], False, stream)
        mdp.check(st, "mdp_create")
        V.zero_()
        st, _ = mdp.mdp_solve(h, eopts, V, pi, stream)
        mdp.check(st, "mdp_solve")
        Vh.copy_(V, non_blocking=True)
        pih.copy_(pi, non_blocking=True)
        torch.cuda.synchronize()
        mdp.mdp_destroy(h)
        if i:  # the first pass is a warm-up
            e2e_times.append(time.perf_counter() - t0)
    e2e = sum(e2e_times) / len(e2e_times) if e2e_times else None
    if e2e is not None:
        e2e = max_over_ranks(e2e, dist, "cuda")

    peak, peak_kind = load_peaks()
    sweeps = totals["bellman_sweeps"]
    bell_ms = totals["bellman_ms"] / sweeps
    bell_gbs = bellman_bytes() / (bell_ms * 1e-3) / 1e9
    inner_gbs = totals["inner_bytes"] / (totals["inner_ms"] * 1e-3) / 1e9 if totals["inner_ms"] > 0 else None
    share_bell = totals["bellman_ms"] / (ms * args.steps)
    roofline = {"bound": "hbm", "kernel": "bellman_kernel (fused SpMV + stage cost + min/argmin + residual)",
                "achieved": bell_gbs, "peak": peak, "unit": "GB/s", "frac": bell_gbs / peak,
                "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs, copy)" if peak_kind == "measured"
                else "fallback 6.8 TB/s", "traffic": sweep_traffic(),
                "bytes_per_launch": bellman_bytes(), "avg_launch_ms": bell_ms,
                "share_of_step": share_bell, "tile_states": tile_states, "sweep_shape": shape_info}
    mv_ms = totals["matvec_ms"] / max(1, totals["matvecs_timed"])
    mv_bytes = totals["matvec_bytes"] / max(1, totals["matvecs_timed"])
    mv_gbs = mv_bytes / (mv_ms * 1e-3) / 1e9 if mv_ms > 0 else None
    roof_mv = {"bound": "hbm", "kernel": "gm_matvec_dots_kernel (policy mat-vec of every FP64 Arnoldi step fused with "
                                         "the classical Gram-Schmidt dots; the largest share of the step among single "
                                         "kernels)",
               "achieved": mv_gbs, "peak": peak, "unit": "GB/s", "frac": mv_gbs / peak if mv_gbs else None,
               "peak_kind": roofline["peak_kind"],
               "traffic": summary_value("gm_matvec_dots_banded_s4e5.txt", "dram_bytes_per_launch",
                                        "krylov_src_sha256_16", krylov_source_sha()),
               # the capture is of step j = 24 (rows + u_j + w + 24 basis vectors)
               "traffic_step": 24, "traffic_step_algorithmic_bytes": S * K_ROW * 12 + S * 16 + 24 * S * 8,
               # bytes of the sampled launches (steps j = 0, 8, 16, 24): rows + u_j + w + j basis vectors
               "bytes_per_launch": mv_bytes, "avg_launch_ms": mv_ms,
               "launches_timed": int(totals["matvecs_timed"]),
               # every Arnoldi step launches one of them; the timed ones are a sample
               "share_of_step": mv_ms * totals["inner_iters_total"] / (ms * args.steps)}
    # the same launches against the FP64 pipe: 2 (k + j + 2) flops per state (row, dots, w)
    mv_tflops = totals["matvec_flops"] / (totals["matvec_ms"] * 1e-3) / 1e12 if totals["matvec_ms"] > 0 else None
    roof_mv["fp64"] = {"bound": "alu", "achieved": mv_tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                       "frac": mv_tflops / FP64_PEAK_TFLOPS if mv_tflops else None,
                       "peak_kind": "derived: 152 SMs x 2 FP64 FMA per clock x 2 flop x 2.07 GHz",
                       "dgemm_tflops": fp64_dgemm_tflops(),
                       "frac_of_dgemm": (mv_tflops / fp64_dgemm_tflops()) if mv_tflops and fp64_dgemm_tflops() else None}
    # the FP64 projection of the sampled steps (u_{j+1} = w - sum c_i u_i and ||u||^2): FP64-pipe bound
    gs_tflops = totals["gs_flops"] / (totals["gs_ms"] * 1e-3) / 1e12 if totals["gs_ms"] > 0 else None
    fp64_peak = FP64_PEAK_TFLOPS
    roof_gs = {"bound": "alu", "kernel": "gm_project_kernel (FP64 classical Gram-Schmidt projection of an Arnoldi "
                                        "step: j + 2 FMA per state; its dots run in the mat-vec kernel)",
               "achieved": gs_tflops, "peak": fp64_peak, "unit": "TFLOP/s",
               "frac": gs_tflops / fp64_peak if gs_tflops else None,
               "peak_kind": "derived: 152 SMs x 2 FP64 FMA per clock x 2 flop x 2.07 GHz (nominal 1.25 TFLOP/s)",
               "traffic": None, "launches_timed": int(totals["gs_timed"]),
               "avg_launch_ms": totals["gs_ms"] / max(1, totals["gs_timed"]),
               "dgemm_tflops": fp64_dgemm_tflops(),
               "frac_of_dgemm": (gs_tflops / fp64_dgemm_tflops()) if gs_tflops and fp64_dgemm_tflops() else None}
    inner_roof = {"phase": "inner GMRES solves (all kernels and host round trips)",
                  "achieved": inner_gbs, "unit": "GB/s", "frac": inner_gbs / peak if inner_gbs else None,
                  "bytes": totals["inner_bytes"] / args.steps, "ms_per_step": totals["inner_ms"] / args.steps}
    mixed = {"what": "same solves, GMRES inner solver with FP32 Arnoldi cycles and FP64 restart residuals "
                     "(MDP_PREC_MIXED); FP64 sweep and stop test",
             "value": mixed_ms / 1e3, "unit": "s", "ms_per_step": mixed_ms,
             "speedup_vs_f64": ms / mixed_ms,
             "outer_per_step": mtot["outer_iters"] / args.steps, "inner_per_step": mtot["inner_iters_total"] / args.steps,
             "inner_ms_per_step": mtot["inner_ms"] / args.steps,
             "inner_GBps": mtot["inner_bytes"] / (mtot["inner_ms"] * 1e-3) / 1e9 if mtot["inner_ms"] > 0 else None,
             "max_final_residual": mtot["final_residual"], "gpu_launches": int(mtot["kernel_launches"]),
             "error": error_statement(Vmx, pimx, mixed_res, GAMMA, K_ROW, gnorm, (V64, pi64))}

    line = {"metric": METRIC, "value": ms / 1e3, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(),
            "roofline": roofline, "roofline_matvec": roof_mv, "roofline_gs": roof_gs, "roofline_inner": inner_roof, "mixed_precision": mixed,
            "mixed_precision_binary16": quant,
            "iterations": {"outer_per_step": totals["outer_iters"] / args.steps,
                           "inner_per_step": totals["inner_iters_total"] / args.steps,
                           "max_final_residual": totals["final_residual"]},
            "e2e": {"value": e2e, "unit": "s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "what": "mdp_create from pinned host CSR (binary64 values) + graph-driven mdp_solve + read back "
                            "of V and pi"},
            "graph_solve": graph_cmp,
            "gpu_launches": int(totals["kernel_launches"]), "clocks": clocks,
            "step_ms": {"min": min(step_ms), "median": statistics.median(step_ms), "max": max(step_ms)}}
    wall = {"main_s": time.perf_counter() - t_main}
    t_sec = time.perf_counter()
    line["small"] = run_small()
    wall["small_s"] = time.perf_counter() - t_sec
    t_sec = time.perf_counter()
    line["mid_batch"] = run_mid_batch()
    wall["mid_batch_s"] = time.perf_counter() - t_sec
    if args.serve > 0:
        t_sec = time.perf_counter()
        line["serving"] = run_serving(args.serve)
        wall["serving_s"] = time.perf_counter() - t_sec
    if args.stress:
        t_sec = time.perf_counter()
        line["bandwidth_stress"] = run_stress()
        wall["bandwidth_stress_s"] = time.perf_counter() - t_sec
    if oracle_child is not None:
        # start the CPU oracle now: the sections below time whole multi-second solves and the
        # arrival-bound serving stream, which one busy host core does not perturb
        oracle_child.stdin.write("go\n")
        oracle_child.stdin.flush()
    if args.pendulum:
        t_sec = time.perf_counter()
        line["pendulum"] = run_pendulum()
        wall["pendulum_s"] = time.perf_counter() - t_sec
    if args.stream > 0 and world == 1:
        t_sec = time.perf_counter()
        line["serving_stream"] = run_serving_stream(args.stream)
        wall["serving_stream_s"] = time.perf_counter() - t_sec
    line["section_wall_s"] = wall
    line["iterations"]["error"] = error_statement(V64, pi64, s64_res, GAMMA, K_ROW, gnorm)
    if oracle_child is not None:
        out, err = oracle_child.communicate()
        try:
            rec = json.loads(out.strip().splitlines()[-1])
            ov = np.load(oracle_npz)
            V_or, pi_or = ov["V"], ov["pi"]
            line["cpu_baseline"] = {
                "value": rec["seconds"], "unit": "s", "cores": 1, "kind": "oracle",
                "sample": ("the whole workload: one FP64 numpy/scipy oracle solve (Algorithm 1, MGS-GMRES(30)) of the "
                           f"same S={S} instance, gamma, tol and alpha, no scaling; run on one host core in a child "
                           f"process during the pendulum and serving-stream sections (after the kernel and end-to-end "
                           f"timings); {rec['info']}"),
                "nproc": rec["nproc"], "cpu_model": rec["cpu_model"]}
            line["iterations"]["error"].update(error_statement(V64, pi64, s64_res, GAMMA, K_ROW, gnorm,
                                                               (V_or, pi_or), "oracle"))
            line["mixed_precision"]["error"].update(error_statement(Vmx, pimx, mixed_res, GAMMA, K_ROW, gnorm,
                                                                    (V_or, pi_or), "oracle"))
        except (ValueError, IndexError, KeyError, OSError) as e:
            line["cpu_baseline"] = {"value": None, "unit": "s", "cores": 1, "kind": "oracle",
                                    "sample": f"oracle child failed: {e}; {err[-400:]}"}
        finally:
            os.unlink(oracle_npz)
        if line["cpu_baseline"].get("value"):
            line["cpu_baseline"]["all_cores"] = cpu_oracle_all_cores()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
