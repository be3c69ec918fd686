"""mdp_solve_small_batch: Algorithm 1 on many small MDPs, one thread-block cluster per
problem, one launch per cluster size.  Each result is certified by the oracle (its
Bellman residual at the returned V bounds ||V - V*||_inf, Sec. II), equals the same
problem solved alone through this entry point bit for bit, and follows the same
outer trace as the oracle's Algorithm 1 on the small random workload."""
import numpy as np
import pytest

from mdpgen import banded_birth_death, maze, pendulum_grid, ragged_sparse, random_sparse
from oracle import mdp_oracle as O
from tests._util import check_policy, q_tolerance

pytestmark = pytest.mark.gpu

# (data, alpha, tol, restart)
PROBLEMS = [
    ("c1_random_s1000_a4_k8", lambda: random_sparse(1000, 4, 8, 0.9, seed=1), 1e-3, 1e-10, 30),
    ("random_s3000_a7_k5", lambda: random_sparse(3000, 7, 5, 0.99, seed=2), 1e-4, 1e-8, 30),
    ("banded_s5000_a20_k33", lambda: banded_birth_death(5000, 20, 16, 0.999), 0.01, 1e-8, 30),
    ("pendulum_40x40_a9", lambda: pendulum_grid(40, 40, 9, 0.99, seed=3), 1e-3, 1e-8, 20),
    ("maze_30x30", lambda: maze(30, 30, 0.2, seed=7, gamma=0.95)[0], 1e-4, 1e-8, 30),
    ("ragged_s700_a5", lambda: ragged_sparse(700, 5, 40, 0.97, seed=11), 1e-3, 1e-9, 12),
    ("one_state", lambda: random_sparse(1, 2, 1, 0.5, seed=6), 1e-3, 1e-12, 5),
    ("one_action", lambda: random_sparse(900, 1, 6, 0.95, seed=12), 1e-3, 1e-9, 30),
    ("s20000_a3_k6", lambda: random_sparse(20000, 3, 6, 0.99, seed=14), 1e-3, 1e-8, 30),
]


def _args(m):
    return (m.S, m.A, m.row_ptr, m.col, m.val, m.g, m.gamma)


def _opts(mdp, m, tol, alpha, restart, max_outer=1000, max_inner=1000):
    o = mdp.mdp_default_opts()
    o.gamma, o.atol_pi, o.alpha, o.gmres_restart = m.gamma, tol, alpha, restart
    o.max_iter_pi, o.max_iter_ksp = max_outer, max_inner
    return o


def _solve(ms, opts):
    import torch

    from paper_2507_22538_gb300 import mdp
    Ms = [mdp.MDP.from_data(m) for m in ms]
    try:
        V = [torch.zeros(m.S, dtype=torch.float64, device="cuda") for m in ms]
        pi = [torch.empty(m.S, dtype=torch.int32, device="cuda") for m in ms]
        st, status, stats = mdp.mdp_solve_small_batch([M.h for M in Ms], opts, V, pi)
        torch.cuda.synchronize()
        mdp.check(st, "mdp_solve_small_batch")
        return status, [v.cpu().numpy() for v in V], [p.cpu().numpy() for p in pi], stats
    finally:
        for M in Ms:
            M.close()


@pytest.fixture(scope="module")
def problems():
    """Each problem at its parity tolerance tol_p = min(tol, 0.5e-8 (1 - gamma) ||V*||), so
    that the certified bound res / (1 - gamma) is below 1e-8 ||V*||."""
    out = []
    for name, make, alpha, tol, restart in PROBLEMS:
        m = make()
        vn = float(np.max(np.abs(O.ipi(*_args(m), tol=tol, alpha=alpha).V)))
        out.append((name, m, alpha, min(tol, 0.5e-8 * (1 - m.gamma) * vn), restart))
    return out


def test_small_batch_certified_by_oracle(problems):
    from paper_2507_22538_gb300 import mdp
    ms = [p[1] for p in problems]
    opts = [_opts(mdp, m, tol, alpha, restart) for _, m, alpha, tol, restart in problems]
    status, Vs, pis, stats = _solve(ms, opts)
    for (name, m, alpha, tol, restart), st, V, pi, s in zip(problems, status, Vs, pis, stats):
        assert st == mdp.MDP_OK and s.converged == 1, (name, st, s.as_dict())
        assert s.final_residual <= tol
        P = O.stacked_matrix(m.S, m.A, m.row_ptr, m.col, m.val)
        Q = O.q_values(P, m.g, m.gamma, V, m.S, m.A)
        qt = q_tolerance(m, V)
        assert float(np.max(np.abs(Q.min(axis=1) - V))) <= tol + qt, name
        bound = (tol + qt) / (1 - m.gamma)
        assert bound <= 1e-8 * (float(np.max(np.abs(V))) - bound), name
        check_policy(pi, Q, qt)
        if m.S <= 2000:
            Vstar, _, _ = O.policy_iteration(*_args(m))
            assert float(np.max(np.abs(V - Vstar))) <= 1e-8 * float(np.max(np.abs(Vstar))), name


def test_small_batch_equals_alone_and_any_order(problems):
    from paper_2507_22538_gb300 import mdp
    ms = [p[1] for p in problems]
    opts = [_opts(mdp, m, tol, alpha, restart) for _, m, alpha, tol, restart in problems]
    status, Vs, pis, stats = _solve(ms, opts)
    r_status, r_V, r_pi, r_stats = _solve(ms[::-1], opts[::-1])
    for i, m in enumerate(ms):
        a_status, a_V, a_pi, a_stats = _solve([m], [opts[i]])
        j = len(ms) - 1 - i
        for st2, V2, pi2, s2 in ((a_status[0], a_V[0], a_pi[0], a_stats[0]), (r_status[j], r_V[j], r_pi[j], r_stats[j])):
            assert st2 == status[i] and np.array_equal(V2, Vs[i]) and np.array_equal(pi2, pis[i]), problems[i][0]
            assert (s2.outer_iters, s2.inner_iters_total, s2.final_residual) == \
                   (stats[i].outer_iters, stats[i].inner_iters_total, stats[i].final_residual)


def test_small_batch_outer_trace_matches_oracle_ipi():
    """The small random workload (S = 1000, A = 4, k = 8, gamma = 0.9, tol 1e-10): the
    same number of evaluations as the oracle's Algorithm 1, inner counts within one per
    evaluation, the same policy."""
    from paper_2507_22538_gb300 import mdp
    m = random_sparse(1000, 4, 8, 0.9, seed=1)
    ref = O.ipi(*_args(m), tol=1e-10, alpha=1e-3, inner="gmres", restart=30)
    status, V, pi, stats = _solve([m], [_opts(mdp, m, 1e-10, 1e-3, 30)])
    assert status[0] == mdp.MDP_OK
    assert stats[0].outer_iters == ref.outer_iters
    assert abs(stats[0].inner_iters_total - sum(ref.inner_iters)) <= ref.outer_iters
    np.testing.assert_allclose(V[0], ref.V, rtol=0, atol=1e-9)
    assert np.array_equal(pi[0], ref.pi)


def test_small_batch_caps_and_numeric():
    """Outer cap: MDP_NOT_CONVERGED with the iterate after that many evaluations, as the
    oracle's capped run; a NaN start vector: MDP_ERR_NUMERIC."""
    import torch

    from paper_2507_22538_gb300 import mdp
    m = random_sparse(500, 4, 8, 0.99, seed=2)
    status, V, _, stats = _solve([m], [_opts(mdp, m, 1e-12, 0.9, 30, max_outer=3, max_inner=1)])
    assert status[0] == mdp.MDP_NOT_CONVERGED and stats[0].outer_iters == 3 and stats[0].converged == 0
    ref = O.ipi(*_args(m), tol=1e-12, alpha=0.9, inner="gmres", max_outer=3, max_inner=1)
    np.testing.assert_allclose(V[0], ref.V, rtol=0, atol=1e-12)
    with mdp.MDP.from_data(m) as M:
        Vn = torch.zeros(m.S, dtype=torch.float64, device="cuda")
        Vn[7] = float("nan")
        pin = torch.empty(m.S, dtype=torch.int32, device="cuda")
        st, status, _ = mdp.mdp_solve_small_batch([M.h], [_opts(mdp, m, 1e-8, 1e-3, 30)], [Vn], [pin])
        torch.cuda.synchronize()
    assert st == mdp.MDP_OK and status[0] == mdp.MDP_ERR_NUMERIC


def test_small_batch_many_problems():
    """A batch larger than the SM count (200 small random MDPs of different sizes,
    actions, row lengths and discounts): every member converges, certified."""
    from paper_2507_22538_gb300 import mdp
    rng = np.random.default_rng(3)
    ms = [random_sparse(int(rng.integers(50, 3000)), int(rng.integers(2, 9)), int(rng.integers(2, 12)),
                        float(rng.choice([0.9, 0.95, 0.99])), seed=100 + i) for i in range(200)]
    opts = [_opts(mdp, m, 1e-9, 1e-3, 30) for m in ms]
    status, Vs, pis, stats = _solve(ms, opts)
    assert all(s == mdp.MDP_OK for s in status)
    for m, V, pi in list(zip(ms, Vs, pis))[::17]:
        P = O.stacked_matrix(m.S, m.A, m.row_ptr, m.col, m.val)
        Q = O.q_values(P, m.g, m.gamma, V, m.S, m.A)
        qt = q_tolerance(m, V)
        assert float(np.max(np.abs(Q.min(axis=1) - V))) <= 1e-9 + qt
        check_policy(pi, Q, qt)


def test_small_batch_rejects_bad_arguments():
    import torch

    from paper_2507_22538_gb300 import mdp
    m = random_sparse(50, 2, 3, 0.9, seed=1)
    big = random_sparse(65537, 1, 1, 0.9, seed=2)
    with mdp.MDP.from_data(m) as M, mdp.MDP.from_data(big) as B:
        V = torch.zeros(m.S, dtype=torch.float64, device="cuda")
        pi = torch.empty(m.S, dtype=torch.int32, device="cuda")
        Vb = torch.zeros(big.S, dtype=torch.float64, device="cuda")
        pib = torch.empty(big.S, dtype=torch.int32, device="cuda")
        o = _opts(mdp, m, 1e-8, 1e-3, 30)
        assert mdp.mdp_solve_small_batch([B.h], [_opts(mdp, big, 1e-8, 1e-3, 30)], [Vb], [pib])[0] == \
            mdp.MDP_ERR_INVALID_ARG
        assert mdp.mdp_solve_small_batch([M.h, M.h], [o, o], [V, V], [pi, pi])[0] == mdp.MDP_ERR_INVALID_ARG
        for field, value in (("inner", mdp.MDP_TFQMR), ("precision", mdp.MDP_PREC_MIXED),
                             ("gmres_refine", mdp.MDP_REFINE_ALWAYS), ("gamma", 1.0), ("gmres_restart", 33)):
            ob = _opts(mdp, m, 1e-8, 1e-3, 30)
            setattr(ob, field, value)
            assert mdp.mdp_solve_small_batch([M.h], [ob], [V], [pi])[0] == mdp.MDP_ERR_INVALID_ARG, field
        st, status, _ = mdp.mdp_solve_small_batch([M.h], [o], [V], [pi])
        torch.cuda.synchronize()
        assert st == mdp.MDP_OK and status[0] == mdp.MDP_OK
