"""Shared helpers for the GPU parity tests (device upload, tolerances)."""
import numpy as np

EPS = np.finfo(np.float64).eps / 2  # unit roundoff of binary64


def to_device(m):
    import torch
    d = dict(row_ptr=torch.from_numpy(m.row_ptr).cuda(), col=torch.from_numpy(m.col).cuda(),
             val=torch.from_numpy(m.val).cuda(), g=torch.from_numpy(m.g).cuda())
    return d


def q_tolerance(m, V):
    """Bound on |Q_gpu - Q_oracle| for one Bellman application.

    Each Q(s, a) = g + gamma * sum_j p_j V_j is a length-k recursive dot
    product: both sides err by at most gamma_{k+2} (|g| + gamma sum |p_j V_j|)
    with gamma_n = n u / (1 - n u) (Higham, Accuracy and Stability, Sec. 3.1),
    so their difference is at most twice that.
    """
    kmax = int(np.max(np.diff(m.row_ptr)))
    n = kmax + 2
    gam = n * EPS / (1 - n * EPS)
    return 2.0 * gam * (float(np.max(np.abs(m.g))) + m.gamma * float(np.max(np.abs(V))))


def check_policy(pi_gpu, Q_oracle, tol):
    """pi_gpu must equal the oracle's lowest argmin wherever the action gap
    exceeds 2 tol; elsewhere its action must be within 2 tol of the minimum."""
    from oracle.mdp_oracle import action_gaps
    S = Q_oracle.shape[0]
    qmin = Q_oracle.min(axis=1)
    sure = action_gaps(Q_oracle) > 2 * tol
    ref = Q_oracle.argmin(axis=1)
    assert np.array_equal(pi_gpu[sure], ref[sure]), np.flatnonzero(pi_gpu[sure] != ref[sure])[:10]
    assert np.all((pi_gpu >= 0) & (pi_gpu < Q_oracle.shape[1]))
    chosen = Q_oracle[np.arange(S), pi_gpu]
    assert np.all(chosen <= qmin + 2 * tol)
