"""Full-size pendulum grid (1000 x 1000 states, A = 9, 4 bilinear entries per row,
gamma = 0.9999, Sec. IV-C), solved to tol = 1e-8 with the Table 1 defaults.

Near-undiscounted and with small per-step moves, this is the hardest of the
workloads for the inner solver (GMRES(30) and TFQMR both need ~80-100 outer
iterations).  The oracle cannot solve it in test time; it certifies the answer
instead: its own Bellman application at the returned V has residual within tol
(so ||V - V*||_inf <= tol / (1 - gamma), Sec. II), and the returned policy is
greedy for V wherever the action gap is resolvable.
"""
import numpy as np
import pytest

from mdpgen import pendulum_grid
from oracle import mdp_oracle as O
from tests._util import check_policy, q_tolerance

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def pendulum():
    return pendulum_grid(1000, 1000, 9, 0.9999, seed=3)


@pytest.mark.parametrize("inner,precision", [(2, 0), (0, 1)], ids=["tfqmr-f64", "gmres-mixed"])
def test_pendulum_full_size_certified(pendulum, inner, precision):
    import torch

    from paper_2507_22538_gb300 import mdp
    m = pendulum
    tol = 1e-8
    with mdp.MDP.from_data(m) as M:
        V, pi, stats, st = M.solve(m.gamma, tol=tol, alpha=1e-4, inner=inner, restart=30, precision=precision)
        torch.cuda.synchronize()
    assert st == mdp.MDP_OK and stats.converged, stats.as_dict()
    Vg, pg = V.cpu().numpy(), pi.cpu().numpy()
    P = O.stacked_matrix(m.S, m.A, m.row_ptr, m.col, m.val)
    Q = O.q_values(P, m.g, m.gamma, Vg, m.S, m.A)
    qt = q_tolerance(m, Vg)
    assert float(np.max(np.abs(Q.min(axis=1) - Vg))) <= tol + qt
    check_policy(pg, Q, qt)
