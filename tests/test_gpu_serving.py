"""Continuous-batching service: requests of different S, A, k and gamma arrive while
others run; each result must equal the same request solved alone (the kernels are
deterministic for a given problem), and each is certified by the oracle."""
import time

import numpy as np
import pytest

from mdpgen import serving_request
from oracle import mdp_oracle as O

pytestmark = pytest.mark.gpu

MIX = dict(s_range=(200, 20_000), a_range=(2, 16), k_range=(4, 32), gammas=(0.9, 0.99, 0.999))


@pytest.mark.parametrize("graph", [True, False], ids=["graph", "stream"])
def test_results_alone_equal_results_in_the_mix(graph):
    """Graph-driven service (the default) and stream-driven service: each result equals
    the request solved alone, and the two drivers give the same bits."""
    from paper_2507_22538_gb300 import mdp
    from paper_2507_22538_gb300.serve import Request, SolveService, latency_summary, solve_alone
    reqs = [Request(i, serving_request(i, seed=17, **MIX), tol=1e-8, alpha=1e-3) for i in range(24)]
    alone = {r.rid: solve_alone(r, graph=graph) for r in reqs}
    other = {r.rid: solve_alone(r, graph=not graph) for r in reqs[:6]}
    for rid, b in other.items():
        assert np.array_equal(alone[rid].V, b.V) and np.array_equal(alone[rid].pi, b.pi)
        assert alone[rid].inner_iters == b.inner_iters
    # a budget that holds only part of the mix at once: admission must wait for memory
    from paper_2507_22538_gb300.serve import device_bytes
    budget = int(3 * max(device_bytes(r.data) for r in reqs))
    svc = SolveService(slots=4, hbm_budget=budget, graph=graph).start()
    rng = np.random.default_rng(0)
    for r in reqs:
        svc.submit(r)
        time.sleep(float(rng.exponential(0.002)))
    res = svc.wait(len(reqs))
    svc.close()
    assert svc.peak_in_flight >= 2  # work from different requests overlapped
    for r in reqs:
        a, b = alone[r.rid], res[r.rid]
        assert a.status == mdp.MDP_OK and b.status == mdp.MDP_OK
        assert np.array_equal(a.V, b.V) and np.array_equal(a.pi, b.pi)
        assert a.outer_iters == b.outer_iters and a.inner_iters == b.inner_iters
    summ = latency_summary(res)
    assert summ["requests"] == len(reqs) and summ["p99_s"] >= summ["p50_s"] > 0


def test_serving_results_certified_by_oracle():
    from paper_2507_22538_gb300 import mdp
    from paper_2507_22538_gb300.serve import Request, SolveService
    from tests._util import check_policy, q_tolerance
    reqs = [Request(i, serving_request(i, seed=23, **MIX), tol=1e-8, alpha=1e-3) for i in range(8)]
    svc = SolveService(slots=3).start()
    for r in reqs:
        svc.submit(r)
    res = svc.wait(len(reqs))
    svc.close()
    for r in reqs:
        m, out = r.data, res[r.rid]
        assert out.status == mdp.MDP_OK
        P = O.stacked_matrix(m.S, m.A, m.row_ptr, m.col, m.val)
        Q = O.q_values(P, m.g, m.gamma, out.V, m.S, m.A)
        qt = q_tolerance(m, out.V)
        assert float(np.max(np.abs(Q.min(axis=1) - out.V))) <= 1e-8 + qt
        check_policy(out.pi, Q, qt)


def test_request_above_budget_is_refused():
    from paper_2507_22538_gb300.serve import Request, SolveService
    svc = SolveService(slots=1, hbm_budget=1 << 20)
    with pytest.raises(ValueError):
        svc.submit(Request(0, serving_request(0, seed=1, **MIX)))


@pytest.mark.parametrize("graph", [True, False], ids=["graph", "stream"])
def test_batched_service_equals_alone(graph):
    """With batch_max > 1 the service solves pending requests of different S, A, k and
    gamma together (mdp_solve_batch: one graph with a branch per request, or lockstep
    launches); each result still equals the request solved alone, bit for bit."""
    from paper_2507_22538_gb300.serve import Request, SolveService, solve_alone
    reqs = [Request(i, serving_request(i, seed=29, **MIX), tol=1e-8, alpha=1e-3) for i in range(16)]
    svc = SolveService(slots=2, batch_max=8, graph=graph).start()
    for r in reqs:
        svc.submit(r)
    res = svc.wait(len(reqs))
    svc.close()
    assert max(svc.batches) > 1
    for r in reqs:
        alone = solve_alone(r)
        out = res[r.rid]
        assert out.status == alone.status
        assert np.array_equal(out.V, alone.V) and np.array_equal(out.pi, alone.pi)
        assert (out.outer_iters, out.inner_iters) == (alone.outer_iters, alone.inner_iters)


def test_cuda_request_generator_matches_numpy():
    """The CUDA draw of the counter-based serving requests against the numpy draw:
    columns and costs bit for bit, probabilities to rounding."""
    from mdpgen import serving_request_philox
    from mdpgen.cuda_gen import serving_request_cuda
    rng = dict(s_range=(300, 4000), a_range=(2, 9), k_range=(4, 64))
    for rid in (0, 3, 99):
        m = serving_request_philox(rid, seed=11, **rng)
        S, A, k, gamma, rp, col, val, g = serving_request_cuda(rid, seed=11, **rng)
        assert (S, A, gamma) == (m.S, m.A, m.gamma)
        assert np.array_equal(rp.cpu().numpy(), m.row_ptr)
        assert np.array_equal(col.cpu().numpy(), m.col)
        assert np.array_equal(g.cpu().numpy(), m.g)
        np.testing.assert_allclose(val.cpu().numpy(), m.val, rtol=1e-13, atol=0)


class DeviceRequest:
    """A counter-based request drawn on the device when the service admits it."""

    def __init__(self, rid, seed, **ranges):
        from mdpgen import request_header
        self.rid, self.seed, self.ranges = rid, seed, ranges
        self.S, self.A, self.k, self.gamma = request_header(rid, seed, **ranges)
        self.nnz, self.kmax = self.S * self.A * self.k, self.k

    def device_arrays(self):
        from mdpgen.cuda_gen import serving_request_cuda
        return serving_request_cuda(self.rid, self.seed, **self.ranges)[4:]


def test_device_drawn_requests_equal_alone_and_certified():
    """Requests drawn on the device at admission, served continuously with and
    without batching: each result equals the request solved alone, and the oracle
    certifies the smaller ones (regenerated on the host by the numpy draw)."""
    from mdpgen import serving_request_philox
    from paper_2507_22538_gb300 import mdp
    from paper_2507_22538_gb300.serve import Request, SolveService, solve_alone
    from tests._util import q_tolerance
    rng = dict(s_range=(300, 30_000), a_range=(2, 12), k_range=(4, 40), gammas=(0.9, 0.99, 0.999))
    reqs = [Request(i, DeviceRequest(i, 17, **rng), tol=1e-8, alpha=1e-3) for i in range(12)]
    alone = {r.rid: solve_alone(r) for r in reqs}
    for batch_max in (1, 4):
        svc = SolveService(slots=2, batch_max=batch_max).start()
        for r in reqs:
            svc.submit(r)
        res = svc.wait(len(reqs))
        svc.close()
        for r in reqs:
            assert res[r.rid].status == mdp.MDP_OK
            assert np.array_equal(res[r.rid].V, alone[r.rid].V) and np.array_equal(res[r.rid].pi, alone[r.rid].pi)
    for r in reqs:
        if r.data.S * r.data.A * r.data.k > 300_000:
            continue
        m = serving_request_philox(r.rid, 17, **rng)
        V = alone[r.rid].V
        P = O.stacked_matrix(m.S, m.A, m.row_ptr, m.col, m.val)
        Q = O.q_values(P, m.g, m.gamma, V, m.S, m.A)
        # the device draw's probabilities differ from the host draw's by rounding, which
        # moves Q by at most a few ulps of gamma * ||V||
        assert float(np.max(np.abs(Q.min(axis=1) - V))) <= 1e-8 + 4 * q_tolerance(m, V)


class FlakyRequest(DeviceRequest):
    """Fails its first `fails` draws with the allocator's out-of-memory error (a
    host-side fault: nothing runs on the GPU)."""

    def __init__(self, rid, seed, fails=1, **ranges):
        super().__init__(rid, seed, **ranges)
        self.fails = fails

    def device_arrays(self):
        import torch
        if self.fails > 0:
            self.fails -= 1
            raise torch.cuda.OutOfMemoryError("injected out-of-memory")
        return super().device_arrays()


def test_out_of_memory_is_retried_while_others_run():
    """A request that runs out of device memory while another is in flight goes back
    to the queue and completes after it; alone, it fails with MDP_ERR_OOM."""
    from paper_2507_22538_gb300 import mdp
    from paper_2507_22538_gb300.serve import Request, SolveService, solve_alone
    big = dict(s_range=(60_000, 60_001), a_range=(8, 8), k_range=(32, 32), gammas=(0.999,))
    small = dict(s_range=(500, 501), a_range=(3, 3), k_range=(5, 5), gammas=(0.9,))
    first = Request(0, DeviceRequest(0, 31, **big), tol=1e-8, alpha=1e-3)
    flaky = Request(1, FlakyRequest(1, 31, fails=1, **small), tol=1e-8, alpha=1e-3)
    svc = SolveService(slots=2).start()
    svc.submit(first)
    import time
    time.sleep(0.002)
    svc.submit(flaky)
    res = svc.wait(2)
    svc.close()
    assert svc.oom_retries == 1
    assert res[0].status == mdp.MDP_OK and res[1].status == mdp.MDP_OK
    ref = solve_alone(Request(1, DeviceRequest(1, 31, **small), tol=1e-8, alpha=1e-3))
    assert np.array_equal(res[1].V, ref.V)
    lone = SolveService(slots=1).start()
    lone.submit(Request(2, FlakyRequest(1, 31, fails=1, **small), tol=1e-8, alpha=1e-3))
    out = lone.wait(1)
    lone.close()
    assert out[2].status == mdp.MDP_ERR_OOM and lone.oom_retries == 0


def test_small_requests_go_to_the_cluster_solver():
    """With small_states set, pending requests of at most that many states are solved
    together by mdp_solve_small_batch (one cluster each); larger ones take the grid
    path.  Every result equals the request solved alone with the same routing, bit for
    bit, and every small one is certified by the oracle."""
    from paper_2507_22538_gb300 import mdp
    from paper_2507_22538_gb300.serve import Request, SolveService, is_small, solve_alone
    from tests._util import check_policy, q_tolerance
    reqs = [Request(i, serving_request(i, seed=31, **MIX), tol=1e-8, alpha=1e-3) for i in range(24)]
    small = 4096
    assert 0 < sum(is_small(r, small) for r in reqs) < len(reqs)
    alone = {r.rid: solve_alone(r, small_states=small) for r in reqs}
    svc = SolveService(slots=2, small_states=small).start()
    for r in reqs:
        svc.submit(r)
    res = svc.wait(len(reqs))
    svc.close()
    assert max(svc.batches) > 1  # small requests shared a launch
    for r in reqs:
        a, b = alone[r.rid], res[r.rid]
        assert a.status == mdp.MDP_OK and b.status == mdp.MDP_OK
        assert np.array_equal(a.V, b.V) and np.array_equal(a.pi, b.pi)
        assert a.outer_iters == b.outer_iters and a.inner_iters == b.inner_iters
        if is_small(r, small):
            m = r.data
            P = O.stacked_matrix(m.S, m.A, m.row_ptr, m.col, m.val)
            Q = O.q_values(P, m.g, m.gamma, b.V, m.S, m.A)
            qt = q_tolerance(m, b.V)
            assert float(np.max(np.abs(Q.min(axis=1) - b.V))) <= 1e-8 + qt
            check_policy(b.pi, Q, qt)
