"""Pins for the FP64 oracle: closed forms, brute force, invariants and identities.

Each check ties the oracle to something other than itself: a hand-derived
solution, enumeration of all A**S policies with dense solves, a textbook BFS,
or a property of the Bellman operator that holds for any MDP (Sec. II).
"""
import collections
import json
import math
import os

import numpy as np
import pytest

from mdpgen import maze, random_sparse, random_value_vector
from oracle import mdp_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _args(m):
    return (m.S, m.A, m.row_ptr, m.col, m.val, m.g, m.gamma)


def _fixture_args(d):
    return (d["S"], d["A"], np.array(d["row_ptr"]), np.array(d["col"]), np.array(d["val"]),
            np.array(d["g"]), d["gamma"])


# ---------------------------------------------------------------- golden closed forms

@pytest.mark.parametrize("name", ["two_state.json", "three_state.json"])
def test_golden_closed_form(name):
    d = _load(name)
    args = _fixture_args(d)
    Vs, ps = np.array(d["V_star"]), np.array(d["pi_star"])
    for inner in ("gmres", "richardson"):
        r = O.ipi(*args, tol=1e-13, alpha=1e-3, inner=inner)
        assert r.converged
        np.testing.assert_allclose(r.V, Vs, rtol=0, atol=1e-12)
        np.testing.assert_array_equal(r.pi, ps)
    V, pi, _ = O.policy_iteration(*args)
    np.testing.assert_allclose(V, Vs, rtol=0, atol=1e-14)
    np.testing.assert_array_equal(pi, ps)
    vi = O.value_iteration(*args, tol=1e-13)
    np.testing.assert_allclose(vi.V, Vs, atol=1e-12)
    Vb, opt, _ = O.brute_force(*args)
    np.testing.assert_allclose(Vb, Vs, atol=1e-14)
    assert tuple(ps) in opt
    if "Q_star" in d:
        P = O.stacked_matrix(d["S"], d["A"], args[2], args[3], args[4])
        Q = O.q_values(P, args[5], d["gamma"], Vs, d["S"], d["A"])
        np.testing.assert_allclose(Q, np.array(d["Q_star"]), atol=1e-15)


def test_constant_cost_closed_form():
    """g = c everywhere: V* = c / (1 - gamma), every action ties, pi* = 0 (lowest index)."""
    m = random_sparse(40, 3, 5, 0.95, seed=11)
    c = 0.37
    g = np.full_like(m.g, c)
    r = O.ipi(m.S, m.A, m.row_ptr, m.col, m.val, g, m.gamma, tol=1e-12, alpha=1e-3)
    np.testing.assert_allclose(r.V, c / (1 - m.gamma), rtol=1e-12)
    # exact ties: dyadic probabilities (rows sum to exactly 1), c = 1/4, gamma = 3/4, V = 1
    q = random_sparse(40, 3, 5, 0.75, seed=11, quant_bits=11)
    P = O.stacked_matrix(q.S, q.A, q.row_ptr, q.col, q.val)
    TV, pi, res = O.bellman(P, np.full_like(q.g, 0.25), 0.75, np.ones(q.S), q.S, q.A)
    assert res == 0.0 and np.all(TV == 1.0)
    assert np.all(pi == 0)


def test_single_action_uniform_closed_form():
    """A = 1 with P = (1/S) 1 1^T: V = g + gamma mean(g) / (1 - gamma)."""
    S, gamma = 17, 0.8
    row_ptr = np.arange(S + 1) * S
    col = np.tile(np.arange(S), S)
    val = np.full(S * S, 1.0 / S)
    g = np.linspace(-1.0, 2.0, S)
    expect = g + gamma * g.mean() / (1 - gamma)
    for inner in ("gmres", "richardson"):
        r = O.ipi(S, 1, row_ptr, col, val, g, gamma, tol=1e-13, alpha=1e-4, inner=inner)
        np.testing.assert_allclose(r.V, expect, atol=1e-12)


def test_single_state_closed_form():
    """S = 1: V* = min_a g(a) / (1 - gamma), pi* = first argmin."""
    A, gamma = 6, 0.97
    g = np.array([0.5, 0.2, 0.9, 0.2, 0.3, 1.0])
    row_ptr = np.arange(A + 1)
    r = O.ipi(1, A, row_ptr, np.zeros(A, dtype=np.int32), np.ones(A), g, gamma, tol=1e-12)
    np.testing.assert_allclose(r.V, [0.2 / (1 - gamma)], rtol=1e-13)
    assert r.pi[0] == 1


def _bfs_distance(H, W, wall, goal_cell):
    dist = np.full(H * W, -1, dtype=np.int64)
    dist[goal_cell] = 0
    q = collections.deque([goal_cell])
    while q:
        c = q.popleft()
        y, x = divmod(c, W)
        for dy, dx in ((-1, 0), (0, 1), (1, 0), (0, -1)):
            ny, nx = y + dy, x + dx
            if 0 <= ny < H and 0 <= nx < W:
                n = ny * W + nx
                if not wall[n] and dist[n] < 0:
                    dist[n] = dist[c] + 1
                    q.append(n)
    return dist


def test_maze_bfs_closed_form():
    """Deterministic maze (Sec. IV-D): V*(s) = goal_cost * gamma**d(s) / (1 - gamma), d = BFS
    distance to the goal; cells cut off from the goal stay put at cost 0 (V* = 0)."""
    H, W = 9, 13
    m, free_idx, goal = maze(H, W, wall_frac=0.25, seed=5, gamma=0.9)
    wall = np.ones(H * W, dtype=bool)
    wall[free_idx] = False
    dist = _bfs_distance(H, W, wall, (H - 1) * W + (W - 1))[free_idx]
    expect = np.where(dist >= 0, -100.0 * m.gamma ** np.maximum(dist, 0) / (1 - m.gamma), 0.0)
    r = O.ipi(*_args(m), tol=1e-11, alpha=1e-4)
    np.testing.assert_allclose(r.V, expect, atol=1e-8)
    Vp, _, _ = O.policy_iteration(*_args(m))
    np.testing.assert_allclose(Vp, expect, atol=1e-10)


# ---------------------------------------------------------------- brute force

@pytest.mark.parametrize("seed", range(6))
def test_brute_force_tiny(seed):
    rng = np.random.default_rng(seed)
    S, A = int(rng.integers(2, 6)), int(rng.integers(1, 4))
    k = int(rng.integers(1, S + 1))
    gamma = float(rng.choice([0.5, 0.9, 0.99]))
    m = random_sparse(S, A, k, gamma, seed=100 + seed)
    Vb, optimal, _ = O.brute_force(*_args(m))
    scale = max(1.0, np.abs(Vb).max())
    for inner in ("gmres", "richardson"):
        r = O.ipi(*_args(m), tol=1e-12 * scale, alpha=1e-3, inner=inner)
        assert r.converged
        np.testing.assert_allclose(r.V, Vb, atol=1e-10 * scale)
        assert tuple(r.pi) in optimal
    Vp, pp, _ = O.policy_iteration(*_args(m))
    np.testing.assert_allclose(Vp, Vb, atol=1e-11 * scale)
    assert tuple(pp) in optimal


# ---------------------------------------------------------------- invariants of T

@pytest.fixture(scope="module")
def mid_mdp():
    return random_sparse(300, 5, 7, 0.93, seed=21)


def test_contraction_monotone_shift(mid_mdp):
    m = mid_mdp
    P = O.stacked_matrix(m.S, m.A, m.row_ptr, m.col, m.val)
    V = random_value_vector(m.S, 1, 3.0)
    Wv = random_value_vector(m.S, 2, 3.0)
    TV, _, _ = O.bellman(P, m.g, m.gamma, V, m.S, m.A)
    TW, _, _ = O.bellman(P, m.g, m.gamma, Wv, m.S, m.A)
    assert np.max(np.abs(TV - TW)) <= m.gamma * np.max(np.abs(V - Wv)) * (1 + 1e-12)
    # monotonicity: V <= V + |W| implies TV <= T(V + |W|)
    TU, _, _ = O.bellman(P, m.g, m.gamma, V + np.abs(Wv), m.S, m.A)
    assert np.all(TV <= TU + 1e-12)
    # row-stochastic shift: T(V + c 1) = TV + gamma c 1
    c = 1.75
    TVc, pic, _ = O.bellman(P, m.g, m.gamma, V + c, m.S, m.A)
    np.testing.assert_allclose(TVc, TV + m.gamma * c, atol=1e-12)


def test_a_posteriori_bound_and_fixed_point(mid_mdp):
    m = mid_mdp
    Vs, ps, hist = O.policy_iteration(*_args(m))
    P = O.stacked_matrix(m.S, m.A, m.row_ptr, m.col, m.val)
    TVs, pis, res = O.bellman(P, m.g, m.gamma, Vs, m.S, m.A)
    assert res <= 1e-13 * max(1, np.abs(Vs).max())  # V* = T V* to the FP64 floor
    np.testing.assert_array_equal(pis, ps)
    for seed in range(3):
        V = random_value_vector(m.S, 10 + seed, 5.0)
        _, _, r = O.bellman(P, m.g, m.gamma, V, m.S, m.A)
        assert np.max(np.abs(V - Vs)) <= r / (1 - m.gamma) * (1 + 1e-9)
    # Howard PI decreases the cost monotonically
    for a, b in zip(hist, hist[1:]):
        assert np.all(b <= a + 1e-10)


# ---------------------------------------------------------------- algorithm identities

def test_richardson_one_step_is_value_iteration(mid_mdp):
    """Table 2: Richardson with one step and omega = 1 is VI."""
    m = mid_mdp
    a = O.ipi(*_args(m), tol=1e-9, alpha=0.5, inner="richardson", max_inner=1, omega=1.0)
    b = O.value_iteration(*_args(m), tol=1e-9)
    assert a.outer_iters == b.outer_iters
    np.testing.assert_allclose(a.V, b.V, atol=1e-11)
    np.testing.assert_array_equal(a.pi, b.pi)


def test_ipi_inner_solves_start_from_V_and_meet_the_forcing_term():
    """Algorithm 1's inexactness rule: the evaluation at V_k starts from theta_0 = V_k
    and stops once ||g_pi - J_pi theta||_2 < alpha ||T V_k - V_k||_inf, pi greedy for
    V_k.  Checked on every outer step of a converged run (V_k taken from runs capped at
    k evaluations), and, for the start, one GMRES step from V_0 against its closed form:
    the least-squares step along r = g_pi - J V_0, V_1 = V_0 + (Jr.r / Jr.Jr) r."""
    m = random_sparse(40, 3, 5, 0.95, seed=13)
    P = O.stacked_matrix(m.S, m.A, m.row_ptr, m.col, m.val)
    alpha = 0.1
    full = O.ipi(*_args(m), tol=1e-10, alpha=alpha)
    assert full.converged and full.outer_iters >= 3
    prev = O.ipi(*_args(m), tol=1e-10, alpha=alpha, max_outer=0).V
    for k in range(full.outer_iters):
        nxt = O.ipi(*_args(m), tol=1e-10, alpha=alpha, max_outer=k + 1).V
        _, pi, res = O.bellman(P, m.g, m.gamma, prev, m.S, m.A)
        assert res == full.residuals[k]
        Ppi, gpi = O.policy_system(P, m.g, pi, m.A)
        assert np.linalg.norm(gpi - O.apply_J(Ppi, m.gamma, nxt)) < alpha * res, k
        prev = nxt
    V0 = random_value_vector(m.S, 4, 5.0)
    one = O.ipi(*_args(m), V0=V0, tol=0.0, alpha=1e-12, max_outer=1, max_inner=1)
    _, pi, _ = O.bellman(P, m.g, m.gamma, V0, m.S, m.A)
    Ppi, gpi = O.policy_system(P, m.g, pi, m.A)
    J = np.eye(m.S) - m.gamma * Ppi.toarray()
    r = gpi - J @ V0
    Jr = J @ r
    np.testing.assert_allclose(one.V, V0 + (Jr @ r) / (Jr @ Jr) * r, rtol=0, atol=1e-12 * np.abs(V0).max())


def test_one_richardson_step_is_policy_operator(mid_mdp):
    m = mid_mdp
    P = O.stacked_matrix(m.S, m.A, m.row_ptr, m.col, m.val)
    V = random_value_vector(m.S, 3, 2.0)
    TV, pi, _ = O.bellman(P, m.g, m.gamma, V, m.S, m.A)
    Ppi, gpi = O.policy_system(P, m.g, pi, m.A)
    out = O.richardson(lambda x: O.apply_J(Ppi, m.gamma, x), gpi, V, 1.0, 0.0, 1)
    assert out.iters == 1
    np.testing.assert_allclose(out.x, TV, atol=1e-13)


def test_unrestarted_gmres_is_exact_in_n_steps():
    m = random_sparse(25, 3, 6, 0.97, seed=5)
    P = O.stacked_matrix(m.S, m.A, m.row_ptr, m.col, m.val)
    pi = np.arange(m.S) % m.A
    Ppi, gpi = O.policy_system(P, m.g, pi, m.A)
    exact = np.linalg.solve(np.eye(m.S) - m.gamma * Ppi.toarray(), gpi)
    out = O.gmres(lambda x: O.apply_J(Ppi, m.gamma, x), gpi, np.zeros(m.S), m.S, 1e-300, m.S)
    assert out.iters <= m.S
    np.testing.assert_allclose(out.x, exact, atol=1e-12 * np.abs(exact).max())
    # the reported residual is the true one
    r = gpi - O.apply_J(Ppi, m.gamma, out.x)
    assert abs(np.linalg.norm(r) - out.res2) <= 1e-15 * max(1, np.linalg.norm(gpi))


def test_gmres_restarted_matches_dense(mid_mdp):
    m = mid_mdp
    P = O.stacked_matrix(m.S, m.A, m.row_ptr, m.col, m.val)
    pi = (np.arange(m.S) * 7) % m.A
    Ppi, gpi = O.policy_system(P, m.g, pi, m.A)
    exact = np.linalg.solve(np.eye(m.S) - m.gamma * Ppi.toarray(), gpi)
    out = O.gmres(lambda x: O.apply_J(Ppi, m.gamma, x), gpi, np.zeros(m.S), 10, 1e-12, 10000)
    assert out.res2 < 1e-12
    np.testing.assert_allclose(out.x, exact, atol=1e-10)


def test_gmres_minimises_the_residual_over_the_krylov_space():
    """k steps of GMRES from x0 give the x in x0 + K_k(J, r0) with the least
    ||b - J x||_2 (the defining property, Saad Sec. 6.5): compared with a least-squares
    solve over an orthonormal basis of the Krylov space built here by repeated
    products and numpy's QR, with no Arnoldi recurrence or Givens rotation; and the
    residual never grows with k."""
    m = random_sparse(30, 3, 6, 0.9, seed=8)
    P = O.stacked_matrix(m.S, m.A, m.row_ptr, m.col, m.val)
    pi = (np.arange(m.S) * 5) % m.A
    Ppi, gpi = O.policy_system(P, m.g, pi, m.A)
    J = np.eye(m.S) - m.gamma * Ppi.toarray()
    x0 = random_value_vector(m.S, 9, 1.0)
    r0 = gpi - J @ x0
    cols, prev = [], np.inf
    for k in range(1, 9):
        v = r0 if not cols else J @ cols[-1]
        cols.append(v / np.linalg.norm(v))
        Q, _ = np.linalg.qr(np.array(cols).T)
        c = np.linalg.lstsq(J @ Q, r0, rcond=None)[0]
        best = float(np.linalg.norm(r0 - J @ Q @ c))
        out = O.gmres(lambda x: O.apply_J(Ppi, m.gamma, x), gpi, x0, k, 0.0, k)
        assert out.iters == k
        assert abs(out.res2 - best) <= 1e-10 * np.linalg.norm(r0), (k, out.res2, best)
        assert out.res2 <= prev * (1 + 1e-12)
        prev = out.res2


def test_beta_vi_and_opi_converge_to_optimum(mid_mdp):
    """beta-VI (Richardson scale beta, one step) and OPI(W) (W steps) reach V* (Table 2)."""
    m = mid_mdp
    Vs, _, _ = O.policy_iteration(*_args(m))
    b = O.ipi(*_args(m), tol=1e-10, alpha=0.5, inner="richardson", max_inner=1, omega=0.8)
    w = O.ipi(*_args(m), tol=1e-10, alpha=1e-9, inner="richardson", max_inner=5)
    for r in (b, w):
        assert r.converged
        assert np.max(np.abs(r.V - Vs)) <= 1e-10 / (1 - m.gamma)


def test_bellman_states_matches_stacked(mid_mdp):
    m = mid_mdp
    P = O.stacked_matrix(m.S, m.A, m.row_ptr, m.col, m.val)
    V = random_value_vector(m.S, 4, 1.0)
    TV, pi, _ = O.bellman(P, m.g, m.gamma, V, m.S, m.A)
    states = np.array([0, 7, 299])
    rows = (states[:, None] * m.A + np.arange(m.A)[None, :]).ravel()
    k = 7
    cols = np.stack([m.col[m.row_ptr[r]:m.row_ptr[r] + k] for r in rows])
    vals = np.stack([m.val[m.row_ptr[r]:m.row_ptr[r] + k] for r in rows])
    Q, tv, p = O.bellman_states(states, cols, vals, m.g[rows], m.gamma, V, m.A)
    np.testing.assert_allclose(tv, TV[states], atol=1e-15)
    np.testing.assert_array_equal(p, pi[states])


def test_action_gaps_hand_computed():
    """The action gap (second-smallest minus smallest Q per state, Eq. 4's margin of
    uniqueness) on hand-computed cases: the three-state fixture at V*, where
    Q(0, .) = (2, 9/11), Q(1, .) = (1, 10/11) and Q(2, .) = (0, 0) give gaps 13/11,
    1/11 and an exact tie 0; unsorted and repeated values; negative costs; and
    A = 1, which has no second action (inf)."""
    d = _load("three_state.json")
    args = _fixture_args(d)
    P = O.stacked_matrix(d["S"], d["A"], args[2], args[3], args[4])
    Q = O.q_values(P, args[5], d["gamma"], np.array(d["V_star"]), d["S"], d["A"])
    np.testing.assert_allclose(Q, [[2.0, 9 / 11], [1.0, 10 / 11], [0.0, 0.0]], rtol=0, atol=1e-15)
    np.testing.assert_allclose(O.action_gaps(Q), [13 / 11, 1 / 11, 0.0], rtol=0, atol=1e-15)
    hand = np.array([[3.0, 1.0, 2.0], [5.0, 5.0, 7.0], [4.0, 2.0, 2.0], [-1.0, -3.0, 0.0], [9.0, 8.5, 0.25]])
    np.testing.assert_array_equal(O.action_gaps(hand), [1.0, 0.0, 0.0, 2.0, 8.25])
    assert np.all(O.action_gaps(np.array([[0.7], [-2.0]])) == np.inf)


def test_check_policy_rejects_a_wrong_policy():
    """The GPU tests' policy check (tests/_util.py) fails a planted wrong action where
    the gap is resolvable and accepts any minimiser at an exact tie."""
    from tests._util import check_policy
    Q = np.array([[2.0, 9 / 11], [1.0, 10 / 11], [0.0, 0.0]])
    check_policy(np.array([1, 1, 0]), Q, 1e-12)
    check_policy(np.array([1, 1, 1]), Q, 1e-12)  # state 2 is a tie: either action is greedy
    with pytest.raises(AssertionError):
        check_policy(np.array([0, 1, 0]), Q, 1e-12)
    with pytest.raises(AssertionError):
        check_policy(np.array([1, 0, 0]), Q, 1e-12)


# ---------------------------------------------------------------- planted mistakes

def _bellman_argmax_ties(P, g, gamma, V, S, A):
    Q = O.q_values(P, g, gamma, V, S, A)
    return Q.min(axis=1), (A - 1 - np.argmin(Q[:, ::-1], axis=1)).astype(np.int32), float(np.max(np.abs(V - Q.min(axis=1))))


def _bellman_transposed(P, g, gamma, V, S, A):
    Q = np.asarray(g).reshape(S, A) + gamma * (P @ V).reshape(A, S).T
    return Q.min(axis=1), Q.argmin(axis=1).astype(np.int32), float(np.max(np.abs(V - Q.min(axis=1))))


def _pins_hold():
    """Run a subset of the pins; True when all pass."""
    try:
        # the direct Krylov pins first: a broken GMRES or TFQMR fails them at once,
        # while the solves below would iterate to their caps with it
        test_unrestarted_gmres_is_exact_in_n_steps()
        test_gmres_minimises_the_residual_over_the_krylov_space()
        test_tfqmr_terminates_in_2n_half_steps()
        test_ipi_inner_solves_start_from_V_and_meet_the_forcing_term()
        test_bellman_states_matches_stacked(random_sparse(300, 5, 7, 0.93, seed=21))
        test_golden_closed_form("two_state.json")
        test_golden_closed_form("three_state.json")
        test_constant_cost_closed_form()
        test_single_state_closed_form()
        for s in range(3):
            test_brute_force_tiny(s)
        test_tfqmr_solves_policy_system()
        test_jacobi_diagonal_and_one_step_identity()
        test_action_gaps_hand_computed()
        test_check_policy_rejects_a_wrong_policy()
    except (AssertionError, pytest.fail.Exception):
        return False
    return True


def _planted(fn, old, new):
    """The oracle's function fn with one piece of its source replaced (a planted mistake)."""
    import inspect
    import textwrap
    src = textwrap.dedent(inspect.getsource(getattr(O, fn)))
    assert src.count(old) == 1, old
    ns = dict(vars(O))
    exec(compile(src.replace(old, new), "<planted>", "exec"), ns)
    return ns[fn]


SOURCE_MUTANTS = {
    "gmres_rotated_rhs_sign": ("gmres", "e[j + 1] = -sn[j] * e[j]", "e[j + 1] = sn[j] * e[j]"),
    "gmres_stale_rotations": ("gmres", "for i in range(j):  # previous rotations",
                              "for i in range(0):  # previous rotations"),
    "gmres_backsub_row": ("gmres", "float(np.dot(H[i, i + 1:jdone], y[i + 1:]))",
                          "float(np.dot(H[i + 1, i + 1:jdone], y[i + 1:]))"),
    "gmres_basis_unnormalised": ("gmres", "Vb[j + 1] = w / hn", "Vb[j + 1] = w"),
    "tfqmr_step_length": ("tfqmr", "eta = c * c * alpha", "eta = c * alpha"),
    "tfqmr_direction_weight": ("tfqmr", "d = yy + (theta * theta * eta / alpha) * d", "d = yy + (theta * eta / alpha) * d"),
    "tfqmr_v_recurrence_sign": ("tfqmr", "v = u1 + beta * (u2 + beta * v)", "v = u1 + beta * (u2 - beta * v)"),
    "tfqmr_tau_update": ("tfqmr", "tau = tau * theta * c", "tau = tau * c"),
    "ipi_fixed_forcing": ("ipi", "out = gmres(mv, gpi, V, restart, alpha * res, max_inner)",
                          "out = gmres(mv, gpi, V, restart, alpha, max_inner)"),
    "ipi_cold_start": ("ipi", "out = gmres(mv, gpi, V, restart, alpha * res, max_inner)",
                       "out = gmres(mv, gpi, np.zeros(S), restart, alpha * res, max_inner)"),
    "sampled_states_action_major": ("bellman_states", "PV.reshape(n, A)", "PV.reshape(A, n).T"),
    "sampled_states_argmax": ("bellman_states", "Q.argmin(axis=1)", "Q.argmax(axis=1)"),
    "richardson_step_sign": ("richardson", "x = x + omega * r", "x = x - omega * r"),
    "richardson_stale_residual": ("richardson", "        r = b - matvec(x)\n        rn = float(np.linalg.norm(r))\n    return",
                                  "        rn = float(np.linalg.norm(r))\n    return"),
    "jacobi_multiplies_by_diagonal": ("jacobi_richardson", "x = x + omega * r / diag", "x = x + omega * r * diag"),
    "jacobi_ignores_diagonal": ("jacobi_richardson", "x = x + omega * r / diag", "x = x + omega * r"),
}


def _q_without_cost(P, g, gamma, V, S, A):
    return gamma * (P @ np.asarray(V, dtype=np.float64)).reshape(S, A)


MUTANTS = ["argmax_ties", "gamma_one", "action_major_layout", "inner_sign", "policy_row_action_major",
           "J_gamma_squared", "evaluation_sign", "jacobi_diagonal_sign", "dropped_cost", "gaps_reversed",
           "gaps_zero", "gaps_inf", "gaps_largest"] + sorted(SOURCE_MUTANTS)


@pytest.mark.filterwarnings("ignore::RuntimeWarning")  # a planted mistake may overflow or divide by zero
@pytest.mark.parametrize("mutant", MUTANTS)
def test_planted_mistakes_are_caught(monkeypatch, mutant):
    """Plausible mistakes planted in the oracle make at least one pin fail: a wrong
    tie-break, discount, layout or sign in the Bellman operator and in J_pi, the
    policy rows taken action-major (pi(s) S + s instead of s A + pi(s)), the policy
    evaluated with the wrong sign, the Jacobi diagonal with the wrong sign, the
    stage cost dropped from Q, and GMRES with a wrong sign in the rotated right-hand
    side, the earlier rotations not applied to a new column, the back substitution
    reading the wrong row of R, or an unnormalised Arnoldi vector, TFQMR with a
    wrong step length, direction weight, v recurrence or tau update, and iPI with a
    fixed inner tolerance instead of alpha times the Bellman residual, or with its
    inner solve started from zero instead of V_k, Richardson stepping against the
    residual or never refreshing it, Jacobi-Richardson multiplying by the diagonal
    or ignoring it, and the sampled-state Bellman step (the full-size checks' oracle)
    with its rows taken action-major or its argmin turned into an argmax."""
    assert _pins_hold()
    if mutant == "argmax_ties":
        monkeypatch.setattr(O, "bellman", _bellman_argmax_ties)
    elif mutant == "gamma_one":
        orig = O.bellman
        monkeypatch.setattr(O, "bellman", lambda P, g, gamma, V, S, A: orig(P, g, min(1.0, gamma * 1.02), V, S, A))
    elif mutant == "action_major_layout":
        monkeypatch.setattr(O, "bellman", _bellman_transposed)
    elif mutant == "inner_sign":
        monkeypatch.setattr(O, "apply_J", lambda Ppi, gamma, x: x + gamma * (Ppi @ x))
    elif mutant == "policy_row_action_major":
        monkeypatch.setattr(O, "policy_rows", lambda pi, A: np.asarray(pi, dtype=np.int64) * np.asarray(pi).size
                            + np.arange(np.asarray(pi).size, dtype=np.int64))
    elif mutant == "J_gamma_squared":
        monkeypatch.setattr(O, "apply_J", lambda Ppi, gamma, x: x - gamma * gamma * (Ppi @ x))
    elif mutant == "evaluation_sign":
        monkeypatch.setattr(O, "evaluate_policy",
                            lambda Ppi, gpi, gamma, dense_limit=5000:
                            np.linalg.solve(np.eye(gpi.size) + gamma * Ppi.toarray(), gpi))
    elif mutant == "jacobi_diagonal_sign":
        monkeypatch.setattr(O, "jacobi_diagonal",
                            lambda Ppi, gamma: 1.0 + gamma * np.asarray(Ppi.diagonal(), dtype=np.float64))
    elif mutant == "dropped_cost":
        monkeypatch.setattr(O, "q_values", _q_without_cost)
    elif mutant == "gaps_reversed":
        monkeypatch.setattr(O, "action_gaps", lambda Q: (lambda p: p[:, 0] - p[:, 1])(np.partition(Q, 1, axis=1))
                            if Q.shape[1] > 1 else np.full(Q.shape[0], np.inf))
    elif mutant == "gaps_zero":
        monkeypatch.setattr(O, "action_gaps", lambda Q: np.zeros(Q.shape[0]))
    elif mutant == "gaps_inf":
        monkeypatch.setattr(O, "action_gaps", lambda Q: np.full(Q.shape[0], np.inf))
    elif mutant == "gaps_largest":
        monkeypatch.setattr(O, "action_gaps", lambda Q: Q.max(axis=1) - Q.min(axis=1))
    elif mutant in SOURCE_MUTANTS:
        fn = SOURCE_MUTANTS[mutant][0]
        monkeypatch.setattr(O, fn, _planted(*SOURCE_MUTANTS[mutant]))
    assert not _pins_hold()


# ---------------------------------------------------------------- TFQMR and Jacobi (Sec. IV-C/D, Table 2)

def test_tfqmr_solves_policy_system():
    """TFQMR reaches the dense solution of (I - gamma P_pi) v = g_pi to its attainable
    accuracy (short recurrences stagnate near 1e-9 relative here), counting half steps."""
    m = random_sparse(200, 3, 6, 0.97, seed=8)
    P = O.stacked_matrix(m.S, m.A, m.row_ptr, m.col, m.val)
    pi = (np.arange(m.S) * 5) % m.A
    Ppi, gpi = O.policy_system(P, m.g, pi, m.A)
    exact = np.linalg.solve(np.eye(m.S) - m.gamma * Ppi.toarray(), gpi)
    mv = lambda x: O.apply_J(Ppi, m.gamma, x)
    bn = float(np.linalg.norm(gpi))
    out = O.tfqmr(mv, gpi, np.zeros(m.S), 1e-8 * bn, 5000)
    assert out.res2 < 1e-7 * bn
    np.testing.assert_allclose(out.x, exact, atol=1e-7 * bn / (1 - m.gamma))
    for cap in (1, 2, 3, 7, 20):
        assert O.tfqmr(mv, gpi, np.zeros(m.S), 0.0, cap).iters == cap
    r10, r40 = (O.tfqmr(mv, gpi, np.zeros(m.S), 0.0, c).res2 for c in (10, 40))
    assert r40 < 1e-3 * r10


def test_tfqmr_terminates_in_2n_half_steps():
    """On an n-state policy system TFQMR, like the BiCG process under it, ends at the
    exact solution once the Krylov space is exhausted: after 2n half steps (n BiCG
    steps, each two products by J) the iterate equals the dense solve to rounding
    level, while two half steps fewer it does not yet (Freund 1993)."""
    for seed in range(5):
        m = random_sparse(6, 3, 4, 0.9, seed=seed)
        P = O.stacked_matrix(m.S, m.A, m.row_ptr, m.col, m.val)
        pi = (np.arange(m.S) * 5) % m.A
        Ppi, gpi = O.policy_system(P, m.g, pi, m.A)
        exact = np.linalg.solve(np.eye(m.S) - m.gamma * Ppi.toarray(), gpi)
        mv = lambda x: O.apply_J(Ppi, m.gamma, x)
        scale = np.abs(exact).max()
        full = O.tfqmr(mv, gpi, np.zeros(m.S), 0.0, 2 * m.S)
        assert full.iters == 2 * m.S
        assert np.abs(full.x - exact).max() <= 1e-12 * scale, seed
        short = O.tfqmr(mv, gpi, np.zeros(m.S), 0.0, 2 * m.S - 2)
        assert np.abs(short.x - exact).max() > 1e-9 * scale, seed


@pytest.mark.parametrize("seed", range(4))
def test_ipi_tfqmr_and_jacobi_match_brute_force(seed):
    rng = np.random.default_rng(50 + seed)
    S, A = int(rng.integers(2, 6)), int(rng.integers(1, 4))
    m = random_sparse(S, A, int(rng.integers(1, S + 1)), float(rng.choice([0.5, 0.9, 0.99])), seed=200 + seed)
    Vb, optimal, _ = O.brute_force(*_args(m))
    scale = max(1.0, np.abs(Vb).max())
    for inner in ("tfqmr", "jacobi"):
        r = O.ipi(*_args(m), tol=1e-12 * scale, alpha=1e-3, inner=inner, max_inner=5000)
        assert r.converged
        np.testing.assert_allclose(r.V, Vb, atol=1e-10 * scale)
        assert tuple(r.pi) in optimal


def test_maze_tfqmr_bfs_closed_form():
    """The maze study's solver choice (TFQMR, Sec. IV-D) on the BFS closed form."""
    H, W = 9, 13
    m, free_idx, goal = maze(H, W, wall_frac=0.25, seed=5, gamma=0.9)
    wall = np.ones(H * W, dtype=bool)
    wall[free_idx] = False
    dist = _bfs_distance(H, W, wall, (H - 1) * W + (W - 1))[free_idx]
    expect = np.where(dist >= 0, -100.0 * m.gamma ** np.maximum(dist, 0) / (1 - m.gamma), 0.0)
    r = O.ipi(*_args(m), tol=1e-11, alpha=1e-4, inner="tfqmr")
    np.testing.assert_allclose(r.V, expect, atol=1e-8)


def test_jacobi_diagonal_and_one_step_identity():
    """J-VI (Table 2): one Jacobi-preconditioned step is x + D^{-1} (T_pi x - x)."""
    m = random_sparse(60, 2, 60, 0.9, seed=3)  # dense rows: every state has a self-transition
    P = O.stacked_matrix(m.S, m.A, m.row_ptr, m.col, m.val)
    pi = np.arange(m.S) % m.A
    Ppi, gpi = O.policy_system(P, m.g, pi, m.A)
    D = O.jacobi_diagonal(Ppi, m.gamma)
    dense = Ppi.toarray()
    np.testing.assert_allclose(D, 1 - m.gamma * np.diag(dense), atol=0)
    x = random_value_vector(m.S, 2, 1.0)
    out = O.jacobi_richardson(lambda v: O.apply_J(Ppi, m.gamma, v), D, gpi, x, 1.0, 0.0, 1)
    np.testing.assert_allclose(out.x, x + (O.policy_operator(Ppi, gpi, m.gamma, x) - x) / D, atol=1e-13)
