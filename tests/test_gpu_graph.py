"""The graph-driven mdp_solve (opts.graph): Algorithm 1 as one CUDA graph with
conditional WHILE/IF nodes, decided on the device.  It runs the kernels of the
stream-driven solve with the same launch shapes, so V, the policy, the iteration
counts, the residual and the work counters must equal the stream-driven solve's
bit for bit (the stream-driven solve is checked against the oracle in
test_gpu_solve.py); one case is also certified against the oracle directly."""
import numpy as np
import pytest

from mdpgen import banded_birth_death, maze, pendulum_grid, random_sparse
from oracle import mdp_oracle as O

pytestmark = pytest.mark.gpu


def _ragged(S, A, seed, kmax=12):
    """Rows of random lengths 1..kmax: the non-uniform sliced layout."""
    from mdpgen import MDPData
    rng = np.random.default_rng(seed)
    lens = rng.integers(1, kmax + 1, size=S * A)
    row_ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    col = np.empty(row_ptr[-1], dtype=np.int32)
    val = np.empty(row_ptr[-1])
    for r in range(S * A):
        c = np.sort(rng.choice(S, size=lens[r], replace=False))
        w = rng.random(lens[r]) + 1e-3
        col[row_ptr[r]:row_ptr[r + 1]] = c
        val[row_ptr[r]:row_ptr[r + 1]] = w / w.sum()
    return MDPData(S, A, row_ptr, col, val, rng.random(S * A), 0.95, f"ragged({S},{A})")


CASES = [
    ("c1_random_s1000_a4_k8", lambda: random_sparse(1000, 4, 8, 0.9, seed=1), 1e-3, 1e-10),
    ("banded_s5000_a20_k33", lambda: banded_birth_death(5000, 20, 16, 0.999), 0.01, 1e-8),
    ("pendulum_40x40_a9", lambda: pendulum_grid(40, 40, 9, 0.99, seed=3), 1e-3, 1e-8),
    ("maze_30x30", lambda: maze(30, 30, 0.2, seed=7, gamma=0.99)[0], 1e-4, 1e-8),
    ("ragged_s700_a5", lambda: _ragged(700, 5, 3), 1e-3, 1e-9),
    ("single_state", lambda: random_sparse(1, 6, 1, 0.5, seed=7), 1e-3, 1e-10),
]

SAME = ("outer_iters", "converged", "inner_iters_total", "final_residual", "bellman_sweeps", "policy_matvecs",
        "vector_reads", "vector_writes", "policy_value_bytes")


def _solve(mdp, M, m, graph, **kw):
    import torch
    V, pi, stats, st = M.solve(m.gamma, graph=graph, **kw)
    torch.cuda.synchronize()
    return V.cpu(), pi.cpu(), stats.as_dict(), st


def _assert_same(a, b):
    import torch
    Va, pa, sa, sta = a
    Vb, pb, sb, stb = b
    assert sta == stb
    assert torch.equal(Va, Vb) or (torch.isnan(Va).all() and torch.isnan(Vb).all())
    assert torch.equal(pa, pb)
    for f in SAME:
        assert sa[f] == sb[f] or (f == "final_residual" and np.isnan(sa[f]) and np.isnan(sb[f])), (f, sa[f], sb[f])
    assert sa["inner_bytes"] == pytest.approx(sb["inner_bytes"], rel=1e-12)


@pytest.mark.parametrize("precision", ["f64", "mixed"])
@pytest.mark.parametrize("name,make,alpha,tol", CASES, ids=[c[0] for c in CASES])
def test_graph_solve_equals_stream_solve(name, make, alpha, tol, precision):
    from paper_2507_22538_gb300 import mdp
    m = make()
    prec = mdp.MDP_PREC_MIXED if precision == "mixed" else mdp.MDP_PREC_F64
    with mdp.MDP.from_data(m) as M:
        ref = _solve(mdp, M, m, False, tol=tol, alpha=alpha, precision=prec)
        got = _solve(mdp, M, m, True, tol=tol, alpha=alpha, precision=prec)
        again = _solve(mdp, M, m, True, tol=tol, alpha=alpha, precision=prec)  # the cached graph
    assert ref[3] == mdp.MDP_OK and ref[2]["converged"] == 1
    _assert_same(ref, got)
    _assert_same(ref, again)


@pytest.mark.parametrize("refine", ["ifneeded", "always"])
def test_graph_solve_with_reorthogonalisation(refine):
    from paper_2507_22538_gb300 import mdp
    m = pendulum_grid(30, 30, 9, 0.99, seed=5)
    code = mdp.MDP_REFINE_IFNEEDED if refine == "ifneeded" else mdp.MDP_REFINE_ALWAYS
    with mdp.MDP.from_data(m) as M:
        ref = _solve(mdp, M, m, False, tol=1e-9, alpha=1e-3, refine=code)
        got = _solve(mdp, M, m, True, tol=1e-9, alpha=1e-3, refine=code)
    _assert_same(ref, got)


@pytest.mark.parametrize("caps", [(3, 1000), (1000, 2), (2, 1), (0, 1000), (1000, 0)],
                         ids=["outer3", "inner2", "outer2_inner1", "outer0", "inner0"])
def test_graph_solve_caps(caps):
    """Iteration caps: MDP_NOT_CONVERGED (or the stalled inner solve) with the same last iterate."""
    from paper_2507_22538_gb300 import mdp
    m = banded_birth_death(3000, 20, 16, 0.999)
    with mdp.MDP.from_data(m) as M:
        kw = dict(tol=1e-10, alpha=1e-3, max_outer=caps[0], max_inner=caps[1])
        ref = _solve(mdp, M, m, False, **kw)
        got = _solve(mdp, M, m, True, **kw)
    _assert_same(ref, got)
    if caps[0] <= 3:
        assert got[3] == mdp.MDP_NOT_CONVERGED and got[2]["outer_iters"] == caps[0]


def test_graph_solve_nan_start():
    """A NaN in V_0 makes the first Bellman residual non-finite: MDP_ERR_NUMERIC on both paths."""
    import torch
    from paper_2507_22538_gb300 import mdp
    m = random_sparse(500, 4, 8, 0.9, seed=2)
    with mdp.MDP.from_data(m) as M:
        out = []
        for graph in (False, True):
            V0 = torch.zeros(m.S, dtype=torch.float64, device="cuda")
            V0[7] = float("nan")
            o = mdp.mdp_default_opts()
            o.gamma, o.graph = m.gamma, int(graph)
            pi = torch.empty(m.S, dtype=torch.int32, device="cuda")
            st, stats = mdp.mdp_solve(M.h, o, V0, pi)
            torch.cuda.synchronize()
            out.append((st, stats.outer_iters, stats.bellman_sweeps))
    assert out[0] == out[1] and out[0][0] == mdp.MDP_ERR_NUMERIC


def test_graph_rebuilt_when_inputs_change():
    """The cached graph bakes in V, pi, gamma and the options: changing any of them
    gives the stream-driven result for the new arguments, and the launch shape
    chosen by mdp_tune is picked up too."""
    import types

    import torch
    from paper_2507_22538_gb300 import mdp
    m = random_sparse(2000, 6, 10, 0.95, seed=9)
    with mdp.MDP.from_data(m) as M:
        for gamma, tol in ((0.95, 1e-9), (0.9, 1e-9), (0.9, 1e-7), (0.99, 1e-8)):
            g = types.SimpleNamespace(gamma=gamma)
            _assert_same(_solve(mdp, M, g, False, tol=tol, alpha=1e-3), _solve(mdp, M, g, True, tol=tol, alpha=1e-3))
        st, ts, ms = mdp.mdp_tune(M.h, 0.9)
        assert st == mdp.MDP_OK
        g = types.SimpleNamespace(gamma=0.9)
        _assert_same(_solve(mdp, M, g, False, tol=1e-9, alpha=1e-3), _solve(mdp, M, g, True, tol=1e-9, alpha=1e-3))
        # a warm start from a caller-owned vector (M.solve clones it: a new V pointer every call)
        V0 = torch.from_numpy(np.linspace(0.0, 3.0, m.S)).cuda()
        r = M.solve(0.9, V0=V0, tol=1e-9, alpha=1e-3)
        q = M.solve(0.9, V0=V0, tol=1e-9, alpha=1e-3, graph=True)
        torch.cuda.synchronize()
        assert torch.equal(r[0], q[0]) and torch.equal(r[1], q[1])


def test_graph_solve_certified_by_oracle():
    """The c1 workload (S = 1000, A = 4, k = 8, gamma = 0.9) solved by the graph to
    1e-10: within 1e-8 relative of Howard policy iteration's V*, greedy policy equal
    where the action gap is resolvable."""
    import torch
    from paper_2507_22538_gb300 import mdp
    m = random_sparse(1000, 4, 8, 0.9, seed=1)
    with mdp.MDP.from_data(m) as M:
        V, pi, stats, st = M.solve(m.gamma, tol=1e-10, alpha=1e-3, graph=True)
        _, _, stats_stream, _ = M.solve(m.gamma, tol=1e-10, alpha=1e-3)
        torch.cuda.synchronize()
    assert st == mdp.MDP_OK and stats.converged == 1
    # the cycles stop after ~13 of 30 steps: the graph skips the rest, the stream path launches them as no-ops
    assert 0 < stats.kernel_launches < stats_stream.kernel_launches
    Vs, ps, _ = O.policy_iteration(m.S, m.A, m.row_ptr, m.col, m.val, m.g, m.gamma)
    Vg = V.cpu().numpy()
    assert float(np.max(np.abs(Vg - Vs))) <= 1e-8 * float(np.max(np.abs(Vs)))
    P = O.stacked_matrix(m.S, m.A, m.row_ptr, m.col, m.val)
    Q = O.q_values(P, m.g, m.gamma, Vs, m.S, m.A)
    sure = O.action_gaps(Q) > 1e-9
    assert np.array_equal(pi.cpu().numpy()[sure], ps[sure])


def test_graph_solve_with_uncapped_iterations():
    """Caps at INT_MAX (no cap in practice): the loop guards, which allow caps + 1 and
    + 2 passes, must not overflow and end a converging solve early."""
    from paper_2507_22538_gb300 import mdp
    m = random_sparse(1000, 4, 8, 0.9, seed=1)
    big = 2**31 - 1
    with mdp.MDP.from_data(m) as M:
        ref = _solve(mdp, M, m, False, tol=1e-10, alpha=1e-3, max_outer=big, max_inner=big)
        got = _solve(mdp, M, m, True, tol=1e-10, alpha=1e-3, max_outer=big, max_inner=big)
    assert ref[3] == mdp.MDP_OK
    _assert_same(ref, got)
