"""mdp_solve_batch: Algorithm 1 on many uneven MDPs in lockstep launches.  Each
problem gets its stand-alone block counts, so its V, policy, iteration counts,
residual and status must equal mdp_solve on it alone bit for bit; one member is
also certified against the oracle's optimum."""
import numpy as np
import pytest

from mdpgen import MDPData, banded_birth_death, maze, pendulum_grid, random_sparse
from oracle import mdp_oracle as O

pytestmark = pytest.mark.gpu


def _ragged(S, A, seed, gamma):
    """Rows of 2..7 entries (odd rows cut to their first half, renormalised): a
    non-uniform sliced layout on both the stacked and the policy side."""
    m = random_sparse(S, A, 7, gamma, seed=seed)
    rp, col, val = [0], [], []
    for r in range(S * A):
        c = m.col[m.row_ptr[r]:m.row_ptr[r + 1]]
        v = m.val[m.row_ptr[r]:m.row_ptr[r + 1]]
        n = 2 + (r * 7919) % 6
        c, v = c[:n], v[:n] / v[:n].sum()
        col.extend(c)
        val.extend(v)
        rp.append(rp[-1] + len(c))
    return MDPData(S, A, np.array(rp, dtype=np.int64), np.array(col, dtype=np.int32), np.array(val), m.g, gamma,
                   f"ragged{S}")


F64, MIXED = 0, 1  # MDP_PREC_F64, MDP_PREC_MIXED

# (data, tol, alpha, restart, max_outer, precision)
PROBLEMS = [
    (lambda: random_sparse(1000, 4, 8, 0.9, seed=1), 1e-10, 1e-3, 30, 1000, F64),
    (lambda: random_sparse(3000, 7, 5, 0.99, seed=2), 1e-8, 1e-4, 30, 1000, F64),
    (lambda: banded_birth_death(5000, 20, 16, 0.999), 1e-8, 0.01, 30, 1000, F64),
    (lambda: pendulum_grid(40, 40, 9, 0.99, seed=3), 1e-8, 1e-3, 20, 1000, F64),
    (lambda: maze(30, 30, 0.2, seed=7, gamma=0.95)[0], 1e-8, 1e-4, 30, 1000, F64),
    (lambda: _ragged(700, 5, 11, 0.97), 1e-9, 1e-3, 12, 1000, F64),
    (lambda: random_sparse(2000, 3, 6, 0.999, seed=5), 1e-8, 1e-3, 30, 2, F64),  # stops at the outer cap
    (lambda: random_sparse(1, 2, 1, 0.5, seed=6), 1e-12, 1e-3, 5, 1000, F64),  # one state
    # mixed precision: binary32 policy values, binary16-exact values, and a ragged one
    (lambda: random_sparse(3000, 7, 5, 0.99, seed=2), 1e-8, 1e-4, 30, 1000, MIXED),
    (lambda: random_sparse(2000, 8, 16, 0.99, seed=8, quant_bits=11), 1e-8, 1e-3, 30, 1000, MIXED),
    (lambda: _ragged(900, 4, 12, 0.99), 1e-8, 1e-3, 16, 1000, MIXED),
]


def _opts(m, tol, alpha, restart, max_outer, precision=F64):
    from paper_2507_22538_gb300 import mdp
    o = mdp.mdp_default_opts()
    o.gamma, o.atol_pi, o.alpha, o.gmres_restart, o.max_iter_pi = m.gamma, tol, alpha, restart, max_outer
    o.precision = precision
    return o


def _alone(m, o):
    import torch

    from paper_2507_22538_gb300 import mdp
    with mdp.MDP.from_data(m) as M:
        V = torch.zeros(m.S, dtype=torch.float64, device="cuda")
        pi = torch.empty(m.S, dtype=torch.int32, device="cuda")
        st, stats = mdp.mdp_solve(M.h, o, V, pi, None)
        torch.cuda.synchronize()
        return st, V.cpu().numpy(), pi.cpu().numpy(), stats


def _batch(ms, opts):
    import torch

    from paper_2507_22538_gb300 import mdp
    Ms = [mdp.MDP.from_data(m) for m in ms]
    try:
        V = [torch.zeros(m.S, dtype=torch.float64, device="cuda") for m in ms]
        pi = [torch.empty(m.S, dtype=torch.int32, device="cuda") for m in ms]
        st, status, stats = mdp.mdp_solve_batch([M.h for M in Ms], opts, V, pi, None)
        torch.cuda.synchronize()
        mdp.check(st, "mdp_solve_batch")
        return status, [v.cpu().numpy() for v in V], [p.cpu().numpy() for p in pi], stats
    finally:
        for M in Ms:
            M.close()


@pytest.fixture(scope="module")
def problems():
    return [(make(), tol, alpha, restart, cap, prec) for make, tol, alpha, restart, cap, prec in PROBLEMS]


def test_batch_equals_alone_bitwise(problems):
    from paper_2507_22538_gb300 import mdp
    ms = [p[0] for p in problems]
    opts = [_opts(*p) for p in problems]
    status, Vb, pib, stats = _batch(ms, opts)
    for i, m in enumerate(ms):
        st, V, pi, s1 = _alone(m, opts[i])
        assert status[i] == st, (m.name, status[i], st)
        assert np.array_equal(Vb[i], V), (m.name, float(np.max(np.abs(Vb[i] - V))))
        assert np.array_equal(pib[i], pi), m.name
        assert stats[i].outer_iters == s1.outer_iters, m.name
        assert stats[i].inner_iters_total == s1.inner_iters_total, m.name
        assert stats[i].bellman_sweeps == s1.bellman_sweeps, m.name
        assert stats[i].final_residual == s1.final_residual, m.name
        assert stats[i].converged == s1.converged, m.name
        assert stats[i].policy_value_bytes == s1.policy_value_bytes, m.name
    assert status[6] == mdp.MDP_NOT_CONVERGED and stats[6].outer_iters == 2
    assert [stats[i].policy_value_bytes for i in (8, 9)] == [4, 2]
    assert all(status[i] == mdp.MDP_OK for i in range(len(ms)) if i != 6)


def test_batch_member_certified_by_oracle(problems):
    """The c1 member (random 1000 x 4 x 8, gamma 0.9, tol 1e-10) against the oracle's
    policy iteration: ||V - V*||_inf <= 1e-8 ||V*||_inf and the optimal policy."""
    ms = [p[0] for p in problems]
    opts = [_opts(*p) for p in problems]
    status, Vb, pib, _ = _batch(ms, opts)
    m = ms[0]
    Vs, ps, _ = O.policy_iteration(m.S, m.A, m.row_ptr, m.col, m.val, m.g, m.gamma)
    assert float(np.max(np.abs(Vb[0] - Vs))) <= 1e-8 * float(np.max(np.abs(Vs)))
    P = O.stacked_matrix(m.S, m.A, m.row_ptr, m.col, m.val)
    Q = O.q_values(P, m.g, m.gamma, Vs, m.S, m.A)
    sure = O.action_gaps(Q) > 1e-9
    assert np.array_equal(pib[0][sure], ps[sure])


def test_batch_deterministic_and_order_free(problems):
    """Two runs give the same bits, and so does the batch in reverse order."""
    ms = [p[0] for p in problems]
    opts = [_opts(*p) for p in problems]
    _, V1, p1, _ = _batch(ms, opts)
    _, V2, p2, _ = _batch(ms[::-1], opts[::-1])
    for a, b in zip(V1, V2[::-1]):
        assert np.array_equal(a, b)
    for a, b in zip(p1, p2[::-1]):
        assert np.array_equal(a, b)


def test_batch_rejects_bad_arguments():
    import torch

    from paper_2507_22538_gb300 import mdp
    m = random_sparse(50, 2, 3, 0.9, seed=1)
    with mdp.MDP.from_data(m) as M:
        V = torch.zeros(m.S, dtype=torch.float64, device="cuda")
        pi = torch.empty(m.S, dtype=torch.int32, device="cuda")
        o = _opts(m, 1e-8, 1e-3, 30, 100)
        st, _, _ = mdp.mdp_solve_batch([M.h, M.h], [o, o], [V, V], [pi, pi])
        assert st == mdp.MDP_ERR_INVALID_ARG  # the same handle twice
        o2 = _opts(m, 1e-8, 1e-3, 30, 100)
        o2.inner = mdp.MDP_TFQMR
        st, _, _ = mdp.mdp_solve_batch([M.h], [o2], [V], [pi])
        assert st == mdp.MDP_ERR_INVALID_ARG
        o3 = _opts(m, 1e-8, 1e-3, 30, 100)
        o3.gamma = 1.0
        st, _, _ = mdp.mdp_solve_batch([M.h], [o3], [V], [pi])
        assert st == mdp.MDP_ERR_INVALID_ARG
        st, _, _ = mdp.mdp_solve_batch([], [], [], [])
        assert st == mdp.MDP_ERR_INVALID_ARG
        # the handle still works afterwards
        st, status, stats = mdp.mdp_solve_batch([M.h], [o], [V], [pi])
        assert st == mdp.MDP_OK and status[0] == mdp.MDP_OK


def _batch_v0(ms, opts, V0=None):
    """The batch from given start vectors (zeros where V0[i] is None)."""
    import torch

    from paper_2507_22538_gb300 import mdp
    Ms = [mdp.MDP.from_data(m) for m in ms]
    try:
        V = []
        for i, m in enumerate(ms):
            v = torch.zeros(m.S, dtype=torch.float64, device="cuda")
            if V0 is not None and V0[i] is not None:
                v.copy_(torch.as_tensor(V0[i], dtype=torch.float64))
            V.append(v)
        pi = [torch.empty(m.S, dtype=torch.int32, device="cuda") for m in ms]
        st, status, stats = mdp.mdp_solve_batch([M.h for M in Ms], opts, V, pi, None)
        torch.cuda.synchronize()
        return st, status, [v.cpu().numpy() for v in V], [p.cpu().numpy() for p in pi], stats
    finally:
        for M in Ms:
            M.close()


def _graph_opts(opts):
    for o in opts:
        o.graph = 1
    return opts


def _same_results(a, b, names):
    st_a, status_a, V_a, pi_a, stats_a = a
    st_b, status_b, V_b, pi_b, stats_b = b
    assert st_a == st_b
    for i, name in enumerate(names):
        assert status_a[i] == status_b[i], (name, status_a[i], status_b[i])
        assert np.array_equal(V_a[i], V_b[i], equal_nan=True), name
        assert np.array_equal(pi_a[i], pi_b[i]), name
        for f in ("outer_iters", "inner_iters_total", "bellman_sweeps", "converged", "policy_value_bytes"):
            assert getattr(stats_a[i], f) == getattr(stats_b[i], f), (name, f)
        ra, rb = stats_a[i].final_residual, stats_b[i].final_residual
        assert ra == rb or (np.isnan(ra) and np.isnan(rb)), name


def test_graph_batch_equals_stream_batch_bitwise(problems):
    """opts.graph on every member: the whole batch as one CUDA graph launch, decided
    on the device, gives every problem the stream-driven batch's results bit for bit
    (and so its stand-alone solve's), in both orders."""
    ms = [p[0] for p in problems]
    names = [m.name for m in ms]
    stream = _batch_v0(ms, [_opts(*p) for p in problems])
    graph = _batch_v0(ms, _graph_opts([_opts(*p) for p in problems]))
    _same_results(stream, graph, names)
    rev = _batch_v0(ms[::-1], _graph_opts([_opts(*p) for p in problems])[::-1])
    _same_results(graph, (rev[0], rev[1][::-1], rev[2][::-1], rev[3][::-1], rev[4][::-1]), names)


@pytest.mark.parametrize("caps", [(0, 1000), (1, 1000), (3, 1000), (1000, 0), (1000, 1), (1000, 7), (2, 5)])
def test_graph_batch_caps(caps):
    """Outer and inner iteration caps, per problem, end the device-side loops where
    the stream-driven batch ends them."""
    max_pi, max_ksp = caps
    ms = [random_sparse(1000, 4, 8, 0.9, seed=1), banded_birth_death(3000, 10, 16, 0.999),
          _ragged(500, 3, 13, 0.99)]
    def opts():
        out = []
        for m, restart, prec in zip(ms, (30, 7, 12), (F64, MIXED, F64)):
            o = _opts(m, 1e-9, 1e-3, restart, max_pi, prec)
            o.max_iter_ksp = max_ksp
            out.append(o)
        return out
    stream = _batch_v0(ms, opts())
    graph = _batch_v0(ms, _graph_opts(opts()))
    _same_results(stream, graph, [m.name for m in ms])


def test_graph_batch_nan_member():
    """A member started from a NaN vector fails with MDP_ERR_NUMERIC after its first
    sweep; the others finish as in the stream-driven batch."""
    from paper_2507_22538_gb300 import mdp
    ms = [random_sparse(1000, 4, 8, 0.9, seed=1), random_sparse(800, 5, 6, 0.99, seed=4)]
    V0 = [None, np.full(800, np.nan)]
    stream = _batch_v0(ms, [_opts(m, 1e-9, 1e-3, 30, 1000) for m in ms], V0)
    graph = _batch_v0(ms, _graph_opts([_opts(m, 1e-9, 1e-3, 30, 1000) for m in ms]), V0)
    _same_results(stream, graph, [m.name for m in ms])
    assert graph[1][0] == mdp.MDP_OK and graph[1][1] == mdp.MDP_ERR_NUMERIC


@pytest.mark.parametrize("make", [lambda: banded_birth_death(40000, 20, 16, 0.999, quant_bits=11),
                                  lambda: random_sparse(40000, 6, 12, 0.99, seed=9, quant_bits=11)],
                         ids=["banded_near_diagonal", "random_far_columns"])
def test_mixed_column_offsets_equal_int32_columns(make):
    """A mixed-precision solve whose policy rows keep 16-bit column offsets (every column
    within 32767 states of its row's state: the banded MDP) or 32-bit columns (random
    columns over 40,000 states) gives the batched solver's results, which always read
    32-bit columns, bit for bit; the oracle's Bellman residual certifies the answer."""
    import torch

    from paper_2507_22538_gb300 import mdp
    from tests._util import q_tolerance
    m = make()
    o = _opts(m, 1e-8, 1e-3, 30, 1000, MIXED)
    st, V, pi, s1 = _alone(m, o)
    status, Vb, pib, stats = _batch([m], [_opts(m, 1e-8, 1e-3, 30, 1000, MIXED)])
    assert st == mdp.MDP_OK and status[0] == mdp.MDP_OK
    assert np.array_equal(V, Vb[0]) and np.array_equal(pi, pib[0])
    assert (s1.outer_iters, s1.inner_iters_total) == (stats[0].outer_iters, stats[0].inner_iters_total)
    P = O.stacked_matrix(m.S, m.A, m.row_ptr, m.col, m.val)
    Q = O.q_values(P, m.g, m.gamma, V, m.S, m.A)
    assert float(np.max(np.abs(Q.min(axis=1) - V))) <= 1e-8 + q_tolerance(m, V)
