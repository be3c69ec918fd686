"""Parity of the policy operator J_pi and the inner solvers (Algorithm 1 steps 4-12)."""
import numpy as np
import pytest

from mdpgen import banded_birth_death, pendulum_grid, ragged_sparse, random_sparse, random_value_vector
from oracle import mdp_oracle as O
from tests._util import EPS, to_device

pytestmark = pytest.mark.gpu

CASES = [
    ("c1_shape", lambda: random_sparse(1000, 4, 8, 0.9, seed=1)),
    ("ragged_tail", lambda: random_sparse(1037, 3, 5, 0.99, seed=2)),
    ("banded", lambda: banded_birth_death(4000, 20, 16, 0.999)),
    ("pendulum", lambda: pendulum_grid(40, 40, 9, 0.9999, seed=3)),
    ("tiny", lambda: random_sparse(5, 2, 3, 0.7, seed=9)),
    # rows of 1..40 entries and a few of 120: the non-uniform policy-row gather and row dot
    ("ragged_rows", lambda: ragged_sparse(1500, 4, 40, 0.99, seed=21)),
    ("ragged_rows_f16_exact", lambda: ragged_sparse(1100, 3, 24, 0.97, seed=22, quant_bits=11)),
]


def _policy(m, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, m.A, size=m.S).astype(np.int32)


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_policy_apply_parity(name, make):
    import torch
    from paper_2507_22538_gb300 import mdp
    m = make()
    P = O.stacked_matrix(m.S, m.A, m.row_ptr, m.col, m.val)
    with mdp.MDP.from_data(m) as M:
        for seed in (0, 1):
            pi = _policy(m, seed)
            x = random_value_vector(m.S, seed + 7, 50.0)
            y = M.policy_apply(m.gamma, torch.from_numpy(pi).cuda(), torch.from_numpy(x).cuda())
            torch.cuda.synchronize()
            Ppi, _ = O.policy_system(P, m.g, pi, m.A)
            yo = O.apply_J(Ppi, m.gamma, x)
            k = int(np.max(np.diff(m.row_ptr))) + 2
            tol = 2 * k * EPS * 2 * np.max(np.abs(x))
            np.testing.assert_allclose(y.cpu().numpy(), yo, rtol=0, atol=tol)


def test_invalid_policy_entries_poison_output():
    import torch
    from paper_2507_22538_gb300 import mdp
    m = random_sparse(200, 4, 3, 0.9, seed=3)
    pi = _policy(m, 1)
    pi[17] = 4
    pi[18] = -1
    with mdp.MDP.from_data(m) as M:
        y = M.policy_apply(0.9, torch.from_numpy(pi).cuda(), torch.ones(m.S, dtype=torch.float64, device="cuda"))
        torch.cuda.synchronize()
        y = y.cpu().numpy()
        assert np.isnan(y[17]) and np.isnan(y[18]) and np.all(np.isfinite(np.delete(y, [17, 18])))


@pytest.mark.parametrize("inner", ["gmres", "richardson", "tfqmr", "jacobi"])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_policy_eval_parity(name, make, inner):
    """Both sides stop on ||g_pi - J_pi v||_2 < tol; the true solution v_pi is at most
    ||J_pi^-1||_inf ||.||_inf <= tol / (1 - gamma) away from each."""
    import torch
    from paper_2507_22538_gb300 import mdp
    m = make()
    P = O.stacked_matrix(m.S, m.A, m.row_ptr, m.col, m.val)
    pi = _policy(m, 3)
    Ppi, gpi = O.policy_system(P, m.g, pi, m.A)
    v0 = np.zeros(m.S)
    bn = float(np.linalg.norm(gpi))
    tol = 1e-9 * bn
    krylov = inner in ("gmres", "tfqmr")
    if inner == "tfqmr":
        tol = 1e-7 * bn  # TFQMR's short recurrences stagnate near 1e-9 relative
    maxit = 3000 if krylov else 200
    code = {"gmres": mdp.MDP_GMRES, "richardson": mdp.MDP_RICHARDSON, "tfqmr": mdp.MDP_TFQMR,
            "jacobi": mdp.MDP_RICHARDSON_JACOBI}[inner]
    with mdp.MDP.from_data(m) as M:
        v, it, res, st = M.policy_eval(m.gamma, torch.from_numpy(pi).cuda(), torch.from_numpy(v0).cuda(),
                                       inner=code, restart=30, tol=tol, max_it=maxit)
        torch.cuda.synchronize()
    v = v.cpu().numpy()
    mv = lambda x: O.apply_J(Ppi, m.gamma, x)
    if inner == "gmres":
        ref = O.gmres(mv, gpi, v0, 30, tol, maxit)
    elif inner == "tfqmr":
        ref = O.tfqmr(mv, gpi, v0, tol, maxit)
    elif inner == "richardson":
        ref = O.richardson(mv, gpi, v0, 1.0, tol, maxit)
    else:
        ref = O.jacobi_richardson(mv, O.jacobi_diagonal(Ppi, m.gamma), gpi, v0, 1.0, tol, maxit)
    true_res = float(np.linalg.norm(gpi - mv(v)))
    if st == mdp.MDP_OK or (inner == "tfqmr" and it < maxit):
        if inner == "tfqmr":  # the stop test bounds the quasi-residual; check the true one loosely
            assert abs(res - true_res) <= 1e-6 * max(true_res, tol)  # reported = true residual
            if ref.res2 >= 10 * tol:
                # the short recurrences lose the true residual on this system in the oracle
                # too (random policy, gamma = 0.9999): both stop on the quasi-residual bound
                assert 0 < it < maxit and 0 < ref.iters < maxit, (it, ref.iters)
                return
            assert true_res < 10 * tol
            assert abs(it - ref.iters) <= 2, (it, ref.iters)
            np.testing.assert_allclose(v, ref.x, rtol=0, atol=20 * tol / (1 - m.gamma))
            return
        assert true_res < tol * (1 + 1e-6) + 64 * EPS * bn
        assert ref.res2 < tol
        assert abs(it - ref.iters) <= 1, (it, ref.iters)
        np.testing.assert_allclose(v, ref.x, rtol=0, atol=2 * (tol + 64 * EPS * bn) / (1 - m.gamma))
    else:
        # the cap was hit on both sides (GMRES(30) stagnates on some random policies at
        # gamma near 1; 200 Richardson steps are too few there)
        assert st == mdp.MDP_NOT_CONVERGED and it == maxit and ref.iters == maxit
        if krylov:  # the reported residual is the true residual of the returned iterate
            assert abs(res - true_res) <= 1e-6 * max(true_res, tol)
        else:  # same recurrence on both sides: same iterate
            scale = max(1.0, float(np.max(np.abs(ref.x))))
            np.testing.assert_allclose(v, ref.x, rtol=0, atol=1e-9 * scale)


def test_richardson_one_step_is_policy_operator():
    import torch
    from paper_2507_22538_gb300 import mdp
    m = random_sparse(900, 6, 7, 0.95, seed=4)
    P = O.stacked_matrix(m.S, m.A, m.row_ptr, m.col, m.val)
    pi = _policy(m, 2)
    Ppi, gpi = O.policy_system(P, m.g, pi, m.A)
    x = random_value_vector(m.S, 4, 3.0)
    with mdp.MDP.from_data(m) as M:
        v, it, res, st = M.policy_eval(m.gamma, torch.from_numpy(pi).cuda(), torch.from_numpy(x).cuda(),
                                       inner=mdp.MDP_RICHARDSON, tol=0.0, max_it=1)
        torch.cuda.synchronize()
    assert it == 1 and st == mdp.MDP_NOT_CONVERGED
    np.testing.assert_allclose(v.cpu().numpy(), O.policy_operator(Ppi, gpi, m.gamma, x), rtol=0, atol=1e-13)
