"""Bandwidth-stress random workload at full size: S = 2e6 states, A = 32 actions, 32
entries per row (2.05e9 entries), Dirichlet(0.5) probabilities quantised to 2^-11
(exact in binary16), costs U[0, 1), gamma = 0.99.  Built on the device by the tensor
port of the generator (numpy would take half an hour).

The oracle checks sampled states from their own rows, copied back from the device
arrays that were handed to mdp_create: one Bellman application matches per state,
and a solved V has a per-state Bellman residual within tol and a greedy policy.
"""
import numpy as np
import pytest

from mdpgen import random_value_vector
from oracle import mdp_oracle as O

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

S, A, K, GAMMA, SEED = 2_000_000, 32, 32, 0.99, 21


@pytest.fixture(scope="module")
def stress():
    import torch

    from mdpgen.torch_gen import random_sparse_device
    from paper_2507_22538_gb300 import mdp
    rp, col, val, g = random_sparse_device(S, A, K, GAMMA, SEED, conc=0.5, quant_bits=11)
    M = mdp.MDP(S, A, rp, col, val, g)
    torch.cuda.synchronize()
    yield M, col, val, g
    M.close()


def _rows(col, val, g, states):
    import torch
    rows = (torch.as_tensor(states, device=col.device)[:, None] * A + torch.arange(A, device=col.device)[None, :])
    rows = rows.reshape(-1)
    idx = (rows[:, None] * K + torch.arange(K, device=col.device)[None, :]).reshape(-1)
    cols = col[idx].reshape(-1, K).cpu().numpy().astype(np.int64)
    vals = val[idx].reshape(-1, K).cpu().numpy()
    return cols, vals, g[rows].cpu().numpy()


def _tolerance(vals, gs, V):
    from tests._util import EPS
    n = K + 2
    gam = n * EPS / (1 - n * EPS)
    return 2.0 * gam * (float(np.max(np.abs(gs))) + GAMMA * float(np.max(np.abs(V))))


def _states(seed):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([[0, 1, S // 2, S - 1], rng.integers(0, S, 2000)]))


def test_stress_sampled_bellman(stress):
    import torch
    from tests._util import check_policy
    M, col, val, g = stress
    V = random_value_vector(S, 13, 10.0)
    TV, pi, res = M.bellman(GAMMA, torch.from_numpy(V).cuda())
    torch.cuda.synchronize()
    states = _states(1)
    cols, vals, gs = _rows(col, val, g, states)
    Q, tv, _ = O.bellman_states(states, cols, vals, gs, GAMMA, V, A)
    tol = _tolerance(vals, gs, V)
    np.testing.assert_allclose(TV.cpu().numpy()[states], tv, rtol=0, atol=tol)
    check_policy(pi.cpu().numpy()[states], Q, tol)
    # the residual is the largest |TV - V| of the returned TV
    assert res.item() == float(torch.max(torch.abs(TV - torch.from_numpy(V).cuda())))


@pytest.mark.parametrize("precision", [0, 1], ids=["f64", "mixed"])
def test_stress_solve(stress, precision):
    import torch
    from tests._util import check_policy
    from paper_2507_22538_gb300 import mdp
    M, col, val, g = stress
    tol = 1e-8
    V, pi, stats, st = M.solve(GAMMA, tol=tol, alpha=1e-4, restart=30, precision=precision)
    torch.cuda.synchronize()
    assert st == mdp.MDP_OK and stats.converged, stats.as_dict()
    if precision == 1:
        assert stats.policy_value_bytes == 2  # the quantised probabilities are exact in binary16
    Vg, pg = V.cpu().numpy(), pi.cpu().numpy()
    states = _states(2)
    cols, vals, gs = _rows(col, val, g, states)
    Q, tv, _ = O.bellman_states(states, cols, vals, gs, GAMMA, Vg, A)
    qt = _tolerance(vals, gs, Vg)
    assert float(np.max(np.abs(tv - Vg[states]))) <= tol + qt
    check_policy(pg[states], Q, qt)


def test_stress_lowp_sweep_bit_identical(stress):
    """The full-size workload through the certified low-precision sweep (binary16 values,
    binary32 screen, binary64 re-evaluation of the candidate rows): TV, policy and
    residual bit for bit those of the binary64 sweep, at a random V and at zero."""
    import torch
    M, col, val, g = stress
    for V in (torch.from_numpy(random_value_vector(S, 17, 10.0)).cuda(),
              torch.zeros(S, dtype=torch.float64, device="cuda")):
        a = M.bellman(GAMMA, V)
        b = M.bellman_lowp(GAMMA, V)
        torch.cuda.synchronize()
        for x, y in zip(a, b):
            assert torch.equal(x.view(torch.int32) if x.dtype == torch.int32 else x.view(torch.int64),
                               y.view(torch.int32) if y.dtype == torch.int32 else y.view(torch.int64))
