"""The certified low-precision Bellman sweep (mdp_bellman_lowp, opts.lowp_sweep):
16-bit values and a binary32 screen with a rigorous rounding bound, binary64
re-evaluation of every row that can attain the minimum.  Its TV, policy and
residual must equal mdp_bellman's bit for bit, and through it the oracle's
(Eq. 3-4, Algorithm 1 steps 2-3); solves that use it must equal the binary64
sweep's solves bit for bit (V, policy, iteration counts, residual)."""
import numpy as np
import pytest

from mdpgen import (MDPData, banded_birth_death, maze, pendulum_grid, ragged_sparse, random_sparse,
                    random_value_vector)
from oracle import mdp_oracle as O
from tests._util import check_policy, q_tolerance

pytestmark = pytest.mark.gpu


def _near_ties(S, A, seed):
    """Every action of a state shares one dyadic row; costs differ by 1e-13 or not at
    all: the binary32 screen cannot tell the actions apart, binary64 must decide."""
    m = random_sparse(S, 1, 6, 0.9, seed=seed, quant_bits=11)
    rows = []
    rp = [0]
    col, val = [], []
    for s in range(S):
        c, v = m.col[m.row_ptr[s]:m.row_ptr[s + 1]], m.val[m.row_ptr[s]:m.row_ptr[s + 1]]
        for a in range(A):
            col.extend(c)
            val.extend(v)
            rp.append(rp[-1] + len(c))
    rng = np.random.default_rng(seed)
    base = rng.random(S)
    g = (base[:, None] + 1e-13 * rng.integers(0, 3, size=(S, A))).ravel()
    return MDPData(S, A, np.array(rp, dtype=np.int64), np.array(col, dtype=np.int32), np.array(val), g, 0.9,
                   "near_ties")


CASES = [
    ("c1_shape_f16", lambda: random_sparse(1000, 4, 8, 0.9, seed=1, quant_bits=11)),
    ("ragged_tail_states_f16", lambda: random_sparse(1037, 3, 5, 0.97, seed=2, quant_bits=11)),
    ("one_action", lambda: random_sparse(777, 1, 6, 0.9, seed=3, quant_bits=11)),
    ("many_actions", lambda: random_sparse(300, 33, 7, 0.99, seed=4, quant_bits=11)),
    ("long_rows", lambda: random_sparse(400, 5, 100, 0.9, seed=5, quant_bits=11)),
    ("k1_deterministic", lambda: random_sparse(2000, 7, 1, 0.8, seed=6)),
    ("single_state", lambda: random_sparse(1, 6, 1, 0.5, seed=7)),
    ("banded_f16", lambda: banded_birth_death(5000, 20, 16, 0.999, quant_bits=11)),
    ("pendulum_bf16", lambda: pendulum_grid(60, 50, 9, 0.9999, seed=3, quant_bits=8)),
    ("maze", lambda: maze(30, 30, 0.2, seed=7, gamma=0.99)[0]),
    ("ragged_rows_f16", lambda: ragged_sparse(900, 6, 40, 0.95, seed=9, quant_bits=11)),
    ("random_a32_k32_f16", lambda: random_sparse(3000, 32, 32, 0.99, seed=4, conc=0.5, quant_bits=11)),
    ("near_ties", lambda: _near_ties(400, 5, 11)),
]


def _bits_equal(a, b):
    import torch
    return torch.equal(a.view(torch.int64), b.view(torch.int64))


def _vectors(m):
    """Value vectors of several magnitudes, plus the ones that defeat a binary32
    screen: entries beyond binary32's range, an Inf and a NaN."""
    scale = 1.0 / (1 - m.gamma)
    out = [random_value_vector(m.S, s, scale) for s in (1, 2)]
    out.append(random_value_vector(m.S, 3, 1e-30))
    out.append(random_value_vector(m.S, 7, 1e-40))  # below binary32's normal range
    big = random_value_vector(m.S, 4, scale)
    big[:: max(1, m.S // 7)] = 3e38 * 10  # beyond binary32's largest finite value
    out.append(big)
    if m.S > 3:
        inf = random_value_vector(m.S, 5, scale)
        inf[m.S // 2] = np.inf
        out.append(inf)
        nan = random_value_vector(m.S, 6, scale)
        nan[m.S // 3] = np.nan
        out.append(nan)
    return out


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_lowp_sweep_equals_binary64_sweep(name, make):
    import torch
    from paper_2507_22538_gb300 import mdp
    m = make()
    with mdp.MDP.from_data(m) as M:
        for V in _vectors(m):
            Vd = torch.from_numpy(V).cuda()
            TV, pi, res = M.bellman(m.gamma, Vd)
            TVl, pil, resl = M.bellman_lowp(m.gamma, Vd)
            torch.cuda.synchronize()
            assert _bits_equal(TV, TVl), (name, float((TV - TVl).abs().nan_to_num(0).max()))
            assert torch.equal(pi, pil), name
            assert _bits_equal(res, resl), (res.item(), resl.item())
        # and against the oracle at a regular vector
        V = _vectors(m)[0]
        TVl, pil, resl = M.bellman_lowp(m.gamma, torch.from_numpy(V).cuda())
        torch.cuda.synchronize()
    P = O.stacked_matrix(m.S, m.A, m.row_ptr, m.col, m.val)
    Q = O.q_values(P, m.g, m.gamma, V, m.S, m.A)
    TVo, _, reso = O.bellman(P, m.g, m.gamma, V, m.S, m.A)
    tol = q_tolerance(m, V)
    np.testing.assert_allclose(TVl.cpu().numpy(), TVo, rtol=0, atol=tol)
    assert abs(resl.item() - reso) <= tol
    check_policy(pil.cpu().numpy(), Q, tol)


def test_lowp_sweep_exact_ties_take_lowest_action():
    """g = 1/4, gamma = 3/4, dyadic rows, V = 1: every Q is exactly 1, every action a
    candidate, the lowest one chosen."""
    import torch
    from paper_2507_22538_gb300 import mdp
    m = random_sparse(1000, 9, 6, 0.75, seed=4, quant_bits=11)
    with mdp.MDP(m.S, m.A, m.row_ptr, m.col, m.val, np.full_like(m.g, 0.25)) as M:
        TV, pi, res = M.bellman_lowp(0.75, torch.ones(m.S, dtype=torch.float64, device="cuda"))
        torch.cuda.synchronize()
        assert torch.all(TV == 1.0) and torch.all(pi == 0) and res.item() == 0.0


def test_lowp_sweep_needs_exact_16_bit_probabilities():
    import torch
    from paper_2507_22538_gb300 import mdp
    m = random_sparse(300, 4, 8, 0.9, seed=1)  # Dirichlet weights: not exact in 16 bits
    with mdp.MDP.from_data(m) as M:
        V = torch.zeros(m.S, dtype=torch.float64, device="cuda")
        TV = torch.empty_like(V)
        pi = torch.empty(m.S, dtype=torch.int32, device="cuda")
        assert mdp.mdp_bellman_lowp(M.h, 0.9, V, TV, pi) == mdp.MDP_ERR_INVALID_ARG
        assert "binary16" in mdp.mdp_last_error()
        # the solve option is ignored there: binary64 sweeps
        _, _, stats, st = M.solve(m.gamma, tol=1e-8, alpha=1e-3, lowp_sweep=True)
        assert st == mdp.MDP_OK and stats.bellman_value_bytes == 8 and stats.bellman_rows_fp64 == 0


def test_lowp_sweep_after_tune_keeps_results():
    import torch
    from paper_2507_22538_gb300 import mdp
    m = random_sparse(3000, 32, 12, 0.95, seed=4, quant_bits=11)
    V = torch.from_numpy(random_value_vector(m.S, 2, 5.0)).cuda()
    with mdp.MDP.from_data(m) as M:
        a = M.bellman_lowp(m.gamma, V)
        st, ts, ms = mdp.mdp_tune(M.h, m.gamma)
        assert st == mdp.MDP_OK
        b = M.bellman_lowp(m.gamma, V)
        c = M.bellman(m.gamma, V)
        torch.cuda.synchronize()
    for x, y, z in zip(a, b, c):
        assert torch.equal(x, y) and torch.equal(x, z)


SOLVES = [
    ("banded_f16", lambda: banded_birth_death(5000, 20, 16, 0.999, quant_bits=11), 0.01, 1e-8),
    ("random_a32_k32_f16", lambda: random_sparse(3000, 32, 32, 0.99, seed=4, conc=0.5, quant_bits=11), 1e-4, 1e-8),
    ("pendulum_bf16", lambda: pendulum_grid(40, 40, 9, 0.99, seed=3, quant_bits=8), 1e-3, 1e-8),
    ("ragged_f16", lambda: ragged_sparse(1200, 5, 40, 0.97, seed=13, quant_bits=11), 1e-3, 1e-8),
]


@pytest.mark.parametrize("graph", [False, True], ids=["stream", "graph"])
@pytest.mark.parametrize("precision", [0, 1], ids=["f64", "mixed"])
@pytest.mark.parametrize("name,make,alpha,tol", SOLVES, ids=[c[0] for c in SOLVES])
def test_solve_with_lowp_sweep_is_bit_identical(name, make, alpha, tol, precision, graph):
    """Algorithm 1 with the low-precision sweep: same V, policy, iteration counts and
    residual as with the binary64 sweep, at least one binary64 row per state and sweep,
    and the result certified by the oracle's Bellman residual."""
    import torch
    from paper_2507_22538_gb300 import mdp
    m = make()
    with mdp.MDP.from_data(m) as M:
        V0, p0, s0, st0 = M.solve(m.gamma, tol=tol, alpha=alpha, precision=precision, graph=graph)
        V1, p1, s1, st1 = M.solve(m.gamma, tol=tol, alpha=alpha, precision=precision, graph=graph, lowp_sweep=True)
        torch.cuda.synchronize()
    assert st0 == st1 == mdp.MDP_OK
    assert _bits_equal(V0, V1) and torch.equal(p0, p1)
    assert (s0.outer_iters, s0.inner_iters_total, s0.bellman_sweeps) == (s1.outer_iters, s1.inner_iters_total,
                                                                        s1.bellman_sweeps)
    assert s0.final_residual == s1.final_residual
    assert s0.bellman_value_bytes == 8 and s1.bellman_value_bytes == 2
    assert m.S * s1.bellman_sweeps <= s1.bellman_rows_fp64 <= m.S * m.A * s1.bellman_sweeps
    Vg = V1.cpu().numpy()
    P = O.stacked_matrix(m.S, m.A, m.row_ptr, m.col, m.val)
    Q = O.q_values(P, m.g, m.gamma, Vg, m.S, m.A)
    qt = q_tolerance(m, Vg)
    assert float(np.max(np.abs(Q.min(axis=1) - Vg))) <= tol + qt
    check_policy(p1.cpu().numpy(), Q, qt)
