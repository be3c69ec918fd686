"""Entry offsets beyond 2^31: a random MDP with S = 2.1e6 states, A = 32 actions and
32 entries per row holds 2.15e9 entries, so the rows of states s >= 2^31 / (A k) =
2,097,152 start past the int32 range in the row pointers and in the sliced layout.
One Bellman application and a solve are checked on sampled states on both sides of
that boundary, from the states' own rows copied back from the arrays handed to
mdp_create (the oracle's per-state Bellman operator, Eq. 3)."""
import numpy as np
import pytest

from mdpgen import random_value_vector
from oracle import mdp_oracle as O

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

S, A, K, GAMMA, SEED = 2_100_000, 32, 32, 0.99, 23
FIRST_BEYOND = (1 << 31) // (A * K)  # first state whose rows start at entry offset >= 2^31


@pytest.fixture(scope="module")
def big():
    import torch

    from mdpgen.torch_gen import random_sparse_device
    from paper_2507_22538_gb300 import mdp
    assert S * A * K > (1 << 31)
    rp, col, val, g = random_sparse_device(S, A, K, GAMMA, SEED, conc=0.5, quant_bits=11)
    assert int(rp[FIRST_BEYOND * A].item()) >= (1 << 31) > int(rp[FIRST_BEYOND * A - 1].item())
    M = mdp.MDP(S, A, rp, col, val, g)
    torch.cuda.synchronize()
    yield M, col, val, g
    M.close()
    del rp, col, val, g
    torch.cuda.empty_cache()


def _rows(col, val, g, states):
    import torch
    rows = (torch.as_tensor(states, device=col.device)[:, None] * A + torch.arange(A, device=col.device)[None, :])
    rows = rows.reshape(-1)
    idx = (rows[:, None] * K + torch.arange(K, device=col.device)[None, :]).reshape(-1)
    return (col[idx].reshape(-1, K).cpu().numpy().astype(np.int64), val[idx].reshape(-1, K).cpu().numpy(),
            g[rows].cpu().numpy())


def _tolerance(gs, V):
    from tests._util import EPS
    n = K + 2
    gam = n * EPS / (1 - n * EPS)
    return 2.0 * gam * (float(np.max(np.abs(gs))) + GAMMA * float(np.max(np.abs(V))))


def _states(seed):
    rng = np.random.default_rng(seed)
    edge = np.arange(FIRST_BEYOND - 40, FIRST_BEYOND + 40)
    return np.unique(np.concatenate([[0, S - 1], edge, rng.integers(FIRST_BEYOND, S, 1500),
                                     rng.integers(0, S, 500)]))


def test_bellman_beyond_int32_offsets(big):
    import torch
    from tests._util import check_policy
    M, col, val, g = big
    V = random_value_vector(S, 17, 10.0)
    TV, pi, res = M.bellman(GAMMA, torch.from_numpy(V).cuda())
    torch.cuda.synchronize()
    states = _states(3)
    cols, vals, gs = _rows(col, val, g, states)
    Q, tv, _ = O.bellman_states(states, cols, vals, gs, GAMMA, V, A)
    tol = _tolerance(gs, V)
    np.testing.assert_allclose(TV.cpu().numpy()[states], tv, rtol=0, atol=tol)
    check_policy(pi.cpu().numpy()[states], Q, tol)
    assert res.item() == float(torch.max(torch.abs(TV - torch.from_numpy(V).cuda())))


def test_solve_beyond_int32_offsets(big):
    """The policy rows of states past the boundary are gathered from offsets >= 2^31;
    the solved V must have a per-state Bellman residual within tol there."""
    import torch
    from tests._util import check_policy
    from paper_2507_22538_gb300 import mdp
    M, col, val, g = big
    tol = 1e-8
    V, pi, stats, st = M.solve(GAMMA, tol=tol, alpha=1e-4, restart=30, graph=True)
    torch.cuda.synchronize()
    assert st == mdp.MDP_OK and stats.converged, stats.as_dict()
    Vg, pg = V.cpu().numpy(), pi.cpu().numpy()
    states = _states(4)
    cols, vals, gs = _rows(col, val, g, states)
    Q, tv, _ = O.bellman_states(states, cols, vals, gs, GAMMA, Vg, A)
    qt = _tolerance(gs, Vg)
    assert float(np.max(np.abs(tv - Vg[states]))) <= tol + qt
    check_policy(pg[states], Q, qt)
