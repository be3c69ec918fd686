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


def test_results_alone_equal_results_in_the_mix():
    from paper_2507_22538_gb300 import mdp
    from paper_2507_22538_gb300.serve import Request, SolveService, latency_summary, solve_alone
    reqs = [Request(i, serving_request(i, seed=17, **MIX), tol=1e-8, alpha=1e-3) for i in range(24)]
    alone = {r.rid: solve_alone(r) for r in reqs}
    # a budget that holds only part of the mix at once: admission must wait for memory
    from paper_2507_22538_gb300.serve import device_bytes
    budget = int(3 * max(device_bytes(r.data) for r in reqs))
    svc = SolveService(slots=4, hbm_budget=budget).start()
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


def test_batched_service_equals_alone():
    """With batch_max > 1 the service solves pending requests of different S, A, k and
    gamma together (mdp_solve_batch); each result still equals the request solved
    alone, bit for bit."""
    from paper_2507_22538_gb300.serve import Request, SolveService, solve_alone
    reqs = [Request(i, serving_request(i, seed=29, **MIX), tol=1e-8, alpha=1e-3) for i in range(16)]
    svc = SolveService(slots=2, batch_max=8).start()
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
