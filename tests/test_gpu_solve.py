"""End-to-end parity of mdp_solve (Algorithm 1) with the oracle's optimal V* and pi*."""
import numpy as np
import pytest

from mdpgen import banded_birth_death, maze, pendulum_grid, ragged_sparse, random_sparse
from oracle import mdp_oracle as O

pytestmark = pytest.mark.gpu


def _args(m):
    return (m.S, m.A, m.row_ptr, m.col, m.val, m.g, m.gamma)


def _check_solution(m, V, pi, Vs, tol_outer):
    """||V - V*||_inf <= 1e-8 ||V*||_inf, and pi equals the oracle's greedy policy
    wherever the action gap at V* exceeds both 1e-9 and the certified band."""
    err = float(np.max(np.abs(V - Vs)))
    assert err <= 1e-8 * float(np.max(np.abs(Vs))), err
    P = O.stacked_matrix(m.S, m.A, m.row_ptr, m.col, m.val)
    Q = O.q_values(P, m.g, m.gamma, Vs, m.S, m.A)
    gap = O.action_gaps(Q)
    band = 2 * m.gamma * tol_outer / (1 - m.gamma) + 1e-9 * float(np.max(np.abs(Vs)))
    sure = gap > max(1e-9, band)
    assert np.array_equal(pi[sure], Q.argmin(axis=1)[sure])
    literal = gap > 1e-9
    return int(np.sum(pi[literal] != Q.argmin(axis=1)[literal]))


SOLVE_CASES = [
    ("c1_random_s1000_a4_k8", lambda: random_sparse(1000, 4, 8, 0.9, seed=1), 1e-3, 1e-10),
    ("banded_s5000_a20_k33", lambda: banded_birth_death(5000, 20, 16, 0.999), 0.01, 1e-8),
    ("pendulum_40x40_a9", lambda: pendulum_grid(40, 40, 9, 0.99, seed=3), 1e-3, 1e-8),
    ("random_s3000_a32_k32", lambda: random_sparse(3000, 32, 32, 0.99, seed=4, conc=0.5, quant_bits=11), 1e-4, 1e-8),
    ("maze_40x40", lambda: maze(40, 40, 0.2, seed=7, gamma=0.99)[0], 1e-4, 1e-8),
    # rows of 1..40 entries (and a few of 120): the non-uniform layouts on both the sweep
    # and the policy side, against the oracle
    ("ragged_s1200_a5_k1to40", lambda: ragged_sparse(1200, 5, 40, 0.97, seed=13), 1e-3, 1e-8),
]


@pytest.mark.parametrize("inner", ["gmres", "richardson"])
@pytest.mark.parametrize("name,make,alpha,tol", SOLVE_CASES, ids=[c[0] for c in SOLVE_CASES])
def test_solve_matches_oracle(name, make, alpha, tol, inner):
    """The GPU's V is certified by the oracle: its Bellman residual at V bounds
    ||V - V*||_inf <= res / (1 - gamma) (Sec. II); the solve runs at the parity
    tolerance tol_p = min(tol, 0.5e-8 (1 - gamma) ||V||) so that this bound is
    below 1e-8 ||V*||.  V is also compared with the oracle's own Algorithm 1 run
    at tol_p, and (small cases) with Howard PI's V*."""
    import torch
    from paper_2507_22538_gb300 import mdp
    from tests._util import check_policy, q_tolerance
    m = make()
    if inner == "richardson" and m.gamma > 0.999:
        pytest.skip("Richardson at gamma = 0.9999 needs ~1e5 sweeps; covered by GMRES")
    loose = O.ipi(*_args(m), tol=tol, alpha=alpha, inner="gmres")
    vn = float(np.max(np.abs(loose.V)))
    tol_p = min(tol, 0.5e-8 * (1 - m.gamma) * vn)
    code = mdp.MDP_GMRES if inner == "gmres" else mdp.MDP_RICHARDSON
    with mdp.MDP.from_data(m) as M:
        V, pi, stats, st = M.solve(m.gamma, tol=tol_p, alpha=alpha, inner=code,
                                   max_inner=1000 if inner == "gmres" else 50,
                                   max_outer=300 if inner == "gmres" else 100000)
        torch.cuda.synchronize()
    assert st == mdp.MDP_OK and stats.converged == 1, stats.as_dict()
    assert stats.final_residual <= tol_p
    Vg, pg = V.cpu().numpy(), pi.cpu().numpy()
    P = O.stacked_matrix(m.S, m.A, m.row_ptr, m.col, m.val)
    Q = O.q_values(P, m.g, m.gamma, Vg, m.S, m.A)
    qt = q_tolerance(m, Vg)
    res_o = float(np.max(np.abs(Q.min(axis=1) - Vg)))
    assert res_o <= tol_p + qt
    bound = (tol_p + qt) / (1 - m.gamma)
    assert bound <= 1e-8 * (float(np.max(np.abs(Vg))) - bound)
    check_policy(pg, Q, qt)  # pi is the greedy policy of the returned V
    ref = O.ipi(*_args(m), V0=loose.V, tol=tol_p, alpha=alpha, inner="gmres")
    assert ref.converged
    assert float(np.max(np.abs(Vg - ref.V))) <= 1e-8 * float(np.max(np.abs(ref.V)))
    if m.S * m.A <= 60000 and m.gamma < 0.999:
        Vs, ps, _ = O.policy_iteration(*_args(m))
        _check_solution(m, Vg, pg, Vs, tol_p)


def test_solve_outer_trace_matches_oracle_ipi():
    """Same Algorithm 1 run on both sides: same number of evaluations, same final policy."""
    import torch
    from paper_2507_22538_gb300 import mdp
    m = random_sparse(1000, 4, 8, 0.9, seed=1)
    ref = O.ipi(*_args(m), tol=1e-10, alpha=1e-3, inner="gmres", restart=30)
    with mdp.MDP.from_data(m) as M:
        V, pi, stats, st = M.solve(m.gamma, tol=1e-10, alpha=1e-3)
        torch.cuda.synchronize()
    assert st == mdp.MDP_OK
    assert stats.outer_iters == ref.outer_iters
    assert abs(stats.inner_iters_total - sum(ref.inner_iters)) <= ref.outer_iters
    np.testing.assert_allclose(V.cpu().numpy(), ref.V, rtol=0, atol=1e-9)
    assert np.array_equal(pi.cpu().numpy(), ref.pi)


def test_value_iteration_configuration():
    """Richardson with one step per evaluation is VI (Table 2): same sweep count as the oracle's VI."""
    import torch
    from paper_2507_22538_gb300 import mdp
    m = random_sparse(800, 5, 6, 0.9, seed=3)
    ref = O.value_iteration(*_args(m), tol=1e-9)
    with mdp.MDP.from_data(m) as M:
        V, pi, stats, st = M.solve(m.gamma, tol=1e-9, alpha=0.5, inner=mdp.MDP_RICHARDSON, max_inner=1)
        torch.cuda.synchronize()
    assert st == mdp.MDP_OK and stats.outer_iters == ref.outer_iters
    np.testing.assert_allclose(V.cpu().numpy(), ref.V, rtol=0, atol=1e-11)


def test_outer_cap_returns_not_converged_with_iterate():
    import torch
    from paper_2507_22538_gb300 import mdp
    m = random_sparse(500, 4, 8, 0.99, seed=2)
    with mdp.MDP.from_data(m) as M:
        V, pi, stats, st = M.solve(m.gamma, tol=1e-12, alpha=0.9, inner=mdp.MDP_RICHARDSON, max_inner=1,
                                   max_outer=3)
        torch.cuda.synchronize()
    assert st == mdp.MDP_NOT_CONVERGED and stats.outer_iters == 3 and not stats.converged
    ref = O.value_iteration(*_args(m), tol=0.0, max_iter=3)
    np.testing.assert_allclose(V.cpu().numpy(), ref.V, rtol=0, atol=1e-12)


def test_warm_start_resumes():
    """V_0 is an input (Algorithm 1): restarting from a converged V takes zero evaluations."""
    import torch
    from paper_2507_22538_gb300 import mdp
    m = random_sparse(1000, 4, 8, 0.9, seed=1)
    with mdp.MDP.from_data(m) as M:
        V, pi, stats, st = M.solve(m.gamma, tol=1e-10, alpha=1e-3)
        V2, pi2, stats2, st2 = M.solve(m.gamma, V0=V, tol=1e-10, alpha=1e-3)
        torch.cuda.synchronize()
    assert stats2.outer_iters == 0 and torch.equal(V, V2) and torch.equal(pi, pi2)


@pytest.mark.parametrize("refine", [0, 1, 2], ids=["never", "ifneeded", "always"])
def test_gram_schmidt_refinement_modes(refine):
    """All three Gram-Schmidt refinement choices reach the oracle-certified V."""
    import torch
    from paper_2507_22538_gb300 import mdp
    from tests._util import check_policy, q_tolerance
    for m, alpha in ((random_sparse(1000, 4, 8, 0.9, seed=1), 1e-3), (banded_birth_death(5000, 20, 16, 0.999), 0.01)):
        tol = 0.5e-8 * (1 - m.gamma) * float(np.max(np.abs(O.ipi(*_args(m), tol=1e-8, alpha=alpha).V)))
        with mdp.MDP.from_data(m) as M:
            V, pi, stats, st = M.solve(m.gamma, tol=tol, alpha=alpha, refine=refine, max_outer=300)
            torch.cuda.synchronize()
        assert st == mdp.MDP_OK, stats.as_dict()
        Vg = V.cpu().numpy()
        P = O.stacked_matrix(m.S, m.A, m.row_ptr, m.col, m.val)
        Q = O.q_values(P, m.g, m.gamma, Vg, m.S, m.A)
        qt = q_tolerance(m, Vg)
        assert float(np.max(np.abs(Q.min(axis=1) - Vg))) <= tol + qt
        check_policy(pi.cpu().numpy(), Q, qt)


@pytest.mark.parametrize("name,make,alpha,tol", [c for c in SOLVE_CASES], ids=[c[0] for c in SOLVE_CASES])
def test_mixed_precision_solve_matches_oracle(name, make, alpha, tol):
    """FP32 Arnoldi cycles with FP64 restart residuals (iterative refinement) reach the
    same oracle-certified V as the FP64 path: the outer stop test stays FP64."""
    import torch
    from paper_2507_22538_gb300 import mdp
    from tests._util import check_policy, q_tolerance
    m = make()
    vn = float(np.max(np.abs(O.ipi(*_args(m), tol=tol, alpha=alpha).V)))
    tol_p = min(tol, 0.5e-8 * (1 - m.gamma) * vn)
    with mdp.MDP.from_data(m) as M:
        V, pi, stats, st = M.solve(m.gamma, tol=tol_p, alpha=alpha, precision=mdp.MDP_PREC_MIXED, max_outer=300)
        V64, _, stats64, _ = M.solve(m.gamma, tol=tol_p, alpha=alpha, max_outer=300)
        torch.cuda.synchronize()
    assert st == mdp.MDP_OK and stats.converged, stats.as_dict()
    Vg = V.cpu().numpy()
    P = O.stacked_matrix(m.S, m.A, m.row_ptr, m.col, m.val)
    Q = O.q_values(P, m.g, m.gamma, Vg, m.S, m.A)
    qt = q_tolerance(m, Vg)
    assert float(np.max(np.abs(Q.min(axis=1) - Vg))) <= tol_p + qt
    bound = (tol_p + qt) / (1 - m.gamma)
    assert bound <= 1e-8 * (float(np.max(np.abs(Vg))) - bound)
    check_policy(pi.cpu().numpy(), Q, qt)
    assert float(np.max(np.abs(Vg - V64.cpu().numpy()))) <= 2 * bound



TFQMR_CASES = [
    ("c1_random_s1000_a4_k8", lambda: random_sparse(1000, 4, 8, 0.9, seed=1), 1e-3, 1e-10),
    ("banded_s5000_a20_k33", lambda: banded_birth_death(5000, 20, 16, 0.999), 0.01, 1e-8),
    ("pendulum_60x60_a9_g0999", lambda: pendulum_grid(60, 60, 9, 0.999, seed=3), 1e-3, 1e-8),
    ("pendulum_40x40_a9_g09999", lambda: pendulum_grid(40, 40, 9, 0.9999, seed=3), 1e-3, 1e-8),
    ("maze_40x40", lambda: maze(40, 40, 0.2, seed=7, gamma=0.99)[0], 1e-4, 1e-8),
]


@pytest.mark.parametrize("name,make,alpha,tol", TFQMR_CASES, ids=[c[0] for c in TFQMR_CASES])
def test_tfqmr_solve_certified_by_oracle(name, make, alpha, tol):
    """iPI with the TFQMR inner solver (the paper's choice for the pendulum and maze,
    Sec. IV-C/D), including pendulum grids where GMRES(30) stalls: the oracle's
    Bellman residual at the returned V certifies it."""
    import torch
    from paper_2507_22538_gb300 import mdp
    from tests._util import check_policy, q_tolerance
    m = make()
    ref = O.ipi(*_args(m), tol=tol, alpha=alpha, inner="tfqmr", max_inner=5000)
    assert ref.converged
    vn = float(np.max(np.abs(ref.V)))
    tol_p = min(tol, 0.5e-8 * (1 - m.gamma) * vn)
    with mdp.MDP.from_data(m) as M:
        V, pi, stats, st = M.solve(m.gamma, tol=tol_p, alpha=alpha, inner=mdp.MDP_TFQMR, max_inner=5000, max_outer=500)
        torch.cuda.synchronize()
    assert st == mdp.MDP_OK and stats.converged, stats.as_dict()
    Vg = V.cpu().numpy()
    P = O.stacked_matrix(m.S, m.A, m.row_ptr, m.col, m.val)
    Q = O.q_values(P, m.g, m.gamma, Vg, m.S, m.A)
    qt = q_tolerance(m, Vg)
    assert float(np.max(np.abs(Q.min(axis=1) - Vg))) <= tol_p + qt
    bound = (tol_p + qt) / (1 - m.gamma)
    assert bound <= 1e-8 * (float(np.max(np.abs(Vg))) - bound)
    check_policy(pi.cpu().numpy(), Q, qt)


def test_maze_bfs_closed_form_on_gpu():
    """GPU iPI (TFQMR) on the maze reproduces V*(s) = -100 gamma^d(s) / (1 - gamma)."""
    import collections
    import torch
    from paper_2507_22538_gb300 import mdp
    H, W = 33, 33
    m, free_idx, goal = maze(H, W, 0.25, seed=11, gamma=0.99)
    wall = np.ones(H * W, dtype=bool)
    wall[free_idx] = False
    dist = np.full(H * W, -1)
    dist[(H - 1) * W + W - 1] = 0
    q = collections.deque([(H - 1) * W + W - 1])
    while q:
        c = q.popleft()
        y, x = divmod(c, W)
        for dy, dx in ((-1, 0), (0, 1), (1, 0), (0, -1)):
            ny, nx = y + dy, x + dx
            if 0 <= ny < H and 0 <= nx < W and not wall[ny * W + nx] and dist[ny * W + nx] < 0:
                dist[ny * W + nx] = dist[c] + 1
                q.append(ny * W + nx)
    d = dist[free_idx]
    expect = np.where(d >= 0, -100.0 * m.gamma ** np.maximum(d, 0) / (1 - m.gamma), 0.0)
    with mdp.MDP.from_data(m) as M:
        V, pi, stats, st = M.solve(m.gamma, tol=1e-9, alpha=1e-4, inner=mdp.MDP_TFQMR, max_inner=5000)
        torch.cuda.synchronize()
    assert st == mdp.MDP_OK
    np.testing.assert_allclose(V.cpu().numpy(), expect, atol=1e-9 / (1 - m.gamma) + 1e-10 * 1e4)


@pytest.mark.parametrize("make", [lambda: random_sparse(1000, 4, 8, 0.9, seed=1),
                                  lambda: banded_birth_death(3000, 20, 16, 0.99)], ids=["c1", "banded"])
def test_jacobi_vi_configuration(make):
    """J-VI (Table 2): Jacobi-preconditioned Richardson, one step per evaluation, against the oracle's run."""
    import torch
    from paper_2507_22538_gb300 import mdp
    m = make()
    ref = O.ipi(*_args(m), tol=1e-9, alpha=0.5, inner="jacobi", max_inner=1, max_outer=100000)
    with mdp.MDP.from_data(m) as M:
        V, pi, stats, st = M.solve(m.gamma, tol=1e-9, alpha=0.5, inner=mdp.MDP_RICHARDSON_JACOBI, max_inner=1,
                                   max_outer=100000)
        torch.cuda.synchronize()
    assert st == mdp.MDP_OK and abs(stats.outer_iters - ref.outer_iters) <= 1
    np.testing.assert_allclose(V.cpu().numpy(), ref.V, rtol=0, atol=1e-9 / (1 - m.gamma))



def _power_of_two_rows(S, A, k, gamma, seed):
    """Probabilities 2^-1, ..., 2^-(k-1), 2^-(k-1) per row (exact in bfloat16, and
    with k = 31 the smallest, 2^-30, is below binary16's range)."""
    from mdpgen import MDPData
    rng = np.random.default_rng(seed)
    R = S * A
    col = np.sort(np.stack([rng.choice(S, size=k, replace=False) for _ in range(R)]), axis=1).astype(np.int32)
    p = np.array([2.0 ** -(i + 1) for i in range(k - 1)] + [2.0 ** -(k - 1)])
    val = np.stack([rng.permutation(p) for _ in range(R)])
    g = rng.random(R)
    return MDPData(S, A, np.arange(R + 1, dtype=np.int64) * k, col.ravel(), val.ravel(), g, gamma)


@pytest.mark.parametrize("storage", ["binary16", "bfloat16", "binary32"])
def test_mixed_precision_narrow_storage(storage):
    """With MDP_PREC_MIXED the policy rows are kept in the narrowest format that holds every
    probability exactly (dyadic inputs, binary16 or bfloat16), else binary32; the result
    is certified by the oracle either way."""
    import torch
    from paper_2507_22538_gb300 import mdp
    from tests._util import check_policy, q_tolerance
    if storage == "binary16":
        m, expect = random_sparse(2000, 6, 16, 0.99, seed=41, quant_bits=11), 2
    elif storage == "bfloat16":
        m, expect = _power_of_two_rows(400, 3, 31, 0.99, seed=42), 2
    else:
        m, expect = random_sparse(2000, 6, 16, 0.99, seed=41), 4
    vn = float(np.max(np.abs(O.ipi(*_args(m), tol=1e-8, alpha=1e-3).V)))
    tol_p = min(1e-8, 0.5e-8 * (1 - m.gamma) * vn)
    with mdp.MDP.from_data(m) as M:
        V, pi, stats, st = M.solve(m.gamma, tol=tol_p, alpha=1e-3, precision=mdp.MDP_PREC_MIXED)
        torch.cuda.synchronize()
    assert st == mdp.MDP_OK and stats.policy_value_bytes == expect, stats.as_dict()
    Vg = V.cpu().numpy()
    P = O.stacked_matrix(m.S, m.A, m.row_ptr, m.col, m.val)
    Q = O.q_values(P, m.g, m.gamma, Vg, m.S, m.A)
    qt = q_tolerance(m, Vg)
    assert float(np.max(np.abs(Q.min(axis=1) - Vg))) <= tol_p + qt
    check_policy(pi.cpu().numpy(), Q, qt)
