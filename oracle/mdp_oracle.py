"""Plain FP64 CPU oracle for inexact policy iteration (iPI) on finite discounted MDPs.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import or run this module.  It shares no code
with the CUDA library: it is a slow, direct transcription of the definitions
in "Inside madupite: Technical Design and Performance" (arXiv 2507.22538):

* Sec. II, Eq. 1-4: the MDP {S, A, P, g, gamma}, the policy cost
  V_pi = g_pi + gamma P_pi V_pi, the Bellman optimality operator
  (TV)(s) = min_a [g(s,a) + gamma sum_s' P(s,s',a) V(s')], the residuals
  r(V) = V - TV and r_pi(V) = V - T_pi V, and greedy policies.
* Eq. 5 (Sec. III-B.2): P flattened row-stacked to an (S*A) x S matrix whose
  row s*A + a is P(s, ., a).
* Sec. III-B.3: the greedy step computes PV (length S*A), views it as S x A,
  scales by gamma, adds g and takes a row-wise argmin; the evaluation step
  applies I - gamma P_pi matrix-free; the inner stop test uses the solver's
  2-norm of the linear residual.
* Algorithm 1: the outer iPI loop, and Table 2: the classical DP methods
  (VI, OPI(W), beta-VI) recovered as Richardson inner solvers.

Library primitives serve as single steps (a sparse matrix-vector product, a
dense LAPACK solve, a dot product); there is no blocking or reordering beyond
the definitions.  Readings where the paper is silent (all 0-based):
* V_0 = 0 when no start vector is given.
* argmin ties go to the lowest action index.
* the returned policy is the greedy policy of the returned value vector.
* the inner solve stops once ||g_pi - J_pi theta||_2 < alpha * ||r(V_k)||_inf;
  ||r_{pi_{k+1}}(V_k)||_inf equals ||r(V_k)||_inf because pi_{k+1} is greedy for V_k.
* N_i and N_o cap the number of inner solver iterations and of policy
  evaluations (a Richardson solve with N_i = 1 takes one step: VI in Table 2).
* GMRES: restarted GMRES(m) with modified Gram-Schmidt Arnoldi and Givens
  rotations (Saad, Iterative Methods for Sparse Linear Systems, Sec. 6.5);
  the residual estimate from the rotations drives the stop test, and the true
  residual is recomputed at each restart and at exit.
"""
from __future__ import annotations

import dataclasses
import itertools
import math

import numpy as np
import scipy.sparse as sp


# --------------------------------------------------------------------------
# data: Eq. 5 and the stage-cost matrix (Sec. II, Sec. III-B.2)
# --------------------------------------------------------------------------

def stacked_matrix(S: int, A: int, row_ptr, col, val) -> sp.csr_matrix:
    """The row-stacked (S*A) x S transition matrix of Eq. 5 (row s*A + a = P(s, ., a))."""
    return sp.csr_matrix((np.asarray(val, dtype=np.float64), np.asarray(col), np.asarray(row_ptr)),
                         shape=(S * A, S))


def dense_tensor(S: int, A: int, row_ptr, col, val) -> np.ndarray:
    """P as an A x S x S array, P[a, s, s'] = P(s, s', a), built entry by entry (Sec. II)."""
    P = np.zeros((A, S, S))
    for s in range(S):
        for a in range(A):
            r = s * A + a
            for j in range(int(row_ptr[r]), int(row_ptr[r + 1])):
                P[a, s, int(col[j])] += float(val[j])
    return P


# --------------------------------------------------------------------------
# operators: Eq. 2-4 and the greedy step of Sec. III-B.3
# --------------------------------------------------------------------------

def q_values(P: sp.csr_matrix, g, gamma: float, V, S: int, A: int) -> np.ndarray:
    """Q(s, a) = g(s, a) + gamma (P V)(s*A + a): compute PV (length S*A), view it as
    S x A, scale by gamma and add g (Sec. III-B.3, the approach madupite adopts)."""
    PV = P @ np.asarray(V, dtype=np.float64)
    return np.asarray(g, dtype=np.float64).reshape(S, A) + gamma * PV.reshape(S, A)


def bellman(P: sp.csr_matrix, g, gamma: float, V, S: int, A: int):
    """Bellman optimality operator (Eq. 3), greedy policy (Eq. 4) and ||r(V)||_inf.

    Returns (TV, pi, res): TV(s) = min_a Q(s, a); pi(s) = the lowest a attaining
    the minimum; res = max_s |V(s) - TV(s)| (r(V) = V - TV, Sec. II).
    """
    Q = q_values(P, g, gamma, V, S, A)
    TV = Q.min(axis=1)
    pi = Q.argmin(axis=1).astype(np.int32)  # numpy returns the first minimiser
    res = float(np.max(np.abs(np.asarray(V) - TV))) if S else 0.0
    return TV, pi, res


def policy_rows(pi, A: int) -> np.ndarray:
    """Row indices s*A + pi(s) of P_pi and g_pi inside Eq. 5 and the cost matrix."""
    pi = np.asarray(pi, dtype=np.int64)
    return np.arange(pi.size, dtype=np.int64) * A + pi


def policy_system(P: sp.csr_matrix, g, pi, A: int):
    """(P_pi, g_pi) of Sec. II: P_pi(s, s') = P(s, s', pi(s)), g_pi(s) = g(s, pi(s))."""
    rows = policy_rows(pi, A)
    return P[rows], np.asarray(g, dtype=np.float64)[rows]


def policy_operator(Ppi, gpi, gamma: float, V) -> np.ndarray:
    """T_pi V = g_pi + gamma P_pi V (right-hand side of Eq. 2)."""
    return gpi + gamma * (Ppi @ V)


def apply_J(Ppi, gamma: float, x) -> np.ndarray:
    """J_pi x = (I - gamma P_pi) x, applied without forming J (matrix shell, Sec. III-B.3)."""
    return x - gamma * (Ppi @ x)


# --------------------------------------------------------------------------
# inner solvers (Algorithm 1 steps 6-12)
# --------------------------------------------------------------------------

@dataclasses.dataclass
class InnerResult:
    x: np.ndarray
    iters: int
    res2: float  # 2-norm of the last residual the solver computed


def richardson(matvec, b, x0, omega: float, tol: float, maxit: int) -> InnerResult:
    """Richardson iteration x <- x + omega (b - J x) (Sec. III-C, Table 2).

    Before each step the residual r = b - J x is formed; the loop stops when
    ||r||_2 < tol or after maxit steps.
    """
    x = np.array(x0, dtype=np.float64, copy=True)
    it = 0
    r = b - matvec(x)
    rn = float(np.linalg.norm(r))
    while rn >= tol and it < maxit:
        x = x + omega * r
        it += 1
        r = b - matvec(x)
        rn = float(np.linalg.norm(r))
    return InnerResult(x, it, rn)


def gmres(matvec, b, x0, restart: int, tol: float, maxit: int) -> InnerResult:
    """Restarted GMRES(restart) with modified Gram-Schmidt Arnoldi (Saad, Sec. 6.5).

    One Arnoldi step counts as one iteration.  Within a cycle the least-squares
    residual |e_{j+1}| obtained from the Givens rotations is the stop test;
    the cycle ends when it drops below tol, when restart steps are done, when
    maxit iterations are reached overall, or on breakdown.  The update
    x += V_j y solves the triangular system R y = e.  The true residual is then
    recomputed; the solve ends if it is below tol or maxit is reached,
    otherwise a new cycle starts from it.
    """
    x = np.array(x0, dtype=np.float64, copy=True)
    n = x.size
    it = 0
    r = b - matvec(x)
    beta = float(np.linalg.norm(r))
    while beta >= tol and it < maxit:
        m = restart
        Vb = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        e = np.zeros(m + 1)
        e[0] = beta
        Vb[0] = r / beta
        jdone = 0
        for j in range(m):
            w = matvec(Vb[j])
            for i in range(j + 1):
                H[i, j] = float(np.dot(w, Vb[i]))
                w = w - H[i, j] * Vb[i]
            hn = float(np.linalg.norm(w))
            H[j + 1, j] = hn
            if hn > 0.0:
                Vb[j + 1] = w / hn
            for i in range(j):  # previous rotations applied to column j
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            d = math.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / d
            sn[j] = H[j + 1, j] / d
            H[j, j] = d
            H[j + 1, j] = 0.0
            e[j + 1] = -sn[j] * e[j]
            e[j] = cs[j] * e[j]
            it += 1
            jdone = j + 1
            if abs(e[j + 1]) < tol or it >= maxit or hn == 0.0:
                break
        y = np.zeros(jdone)
        for i in range(jdone - 1, -1, -1):  # back substitution R y = e
            y[i] = (e[i] - float(np.dot(H[i, i + 1:jdone], y[i + 1:]))) / H[i, i]
        x = x + Vb[:jdone].T @ y
        r = b - matvec(x)
        beta = float(np.linalg.norm(r))
    return InnerResult(x, it, beta)


def tfqmr(matvec, b, x0, tol: float, maxit: int) -> InnerResult:
    """Transpose-free QMR (Freund, SIAM J. Sci. Comput. 1993), the inner solver the
    paper uses for the pendulum and maze studies (Sec. IV-C, IV-D).

    Each outer step m forms two Krylov directions (y1, y2) with two products by J
    and takes two quasi-minimal-residual half steps.  One half step (one product
    by J) counts as one iteration.  tau sqrt(k+1) bounds ||b - J x_k||_2 after half
    step k (k = 1, 2, ...); the solve stops once that bound drops below tol, at
    maxit half steps, or when rho or sigma vanish.  Returns the true residual
    norm of the final iterate.
    """
    x = np.array(x0, dtype=np.float64, copy=True)
    r = b - matvec(x)
    tau = float(np.linalg.norm(r))
    if tau < tol or maxit <= 0:
        return InnerResult(x, 0, tau)
    rt = r.copy()
    w = r.copy()
    y1 = r.copy()
    v = matvec(y1)
    u1 = v.copy()
    d = np.zeros_like(x)
    theta = eta = 0.0
    rho = float(np.dot(rt, r))
    k = 0
    while k < maxit:
        sigma = float(np.dot(rt, v))
        if sigma == 0.0 or rho == 0.0:
            break
        alpha = rho / sigma
        y2 = y1 - alpha * v
        u2 = matvec(y2)
        done = False
        for half in (1, 2):
            k += 1
            yy, uu = (y1, u1) if half == 1 else (y2, u2)
            w = w - alpha * uu
            d = yy + (theta * theta * eta / alpha) * d
            theta = float(np.linalg.norm(w)) / tau
            c = 1.0 / math.sqrt(1.0 + theta * theta)
            tau = tau * theta * c
            eta = c * c * alpha
            x = x + eta * d
            if tau * math.sqrt(k + 1) < tol or k >= maxit:
                done = True
                break
        if done:
            break
        rho_new = float(np.dot(rt, w))
        beta = rho_new / rho
        rho = rho_new
        y1 = w + beta * y2
        u1 = matvec(y1)
        v = u1 + beta * (u2 + beta * v)
    return InnerResult(x, k, float(np.linalg.norm(b - matvec(x))))


def jacobi_richardson(matvec, diag, b, x0, omega: float, tol: float, maxit: int) -> InnerResult:
    """Richardson with the Jacobi preconditioner D = diag(I - gamma P_pi) (Table 2, J-VI):
    x <- x + omega D^{-1} (b - J x), stopping on the unpreconditioned ||b - J x||_2 < tol."""
    x = np.array(x0, dtype=np.float64, copy=True)
    it = 0
    r = b - matvec(x)
    rn = float(np.linalg.norm(r))
    while rn >= tol and it < maxit:
        x = x + omega * r / diag
        it += 1
        r = b - matvec(x)
        rn = float(np.linalg.norm(r))
    return InnerResult(x, it, rn)


def jacobi_diagonal(Ppi, gamma: float) -> np.ndarray:
    """Diagonal of J_pi = I - gamma P_pi: 1 - gamma P(s, s, pi(s))."""
    return 1.0 - gamma * np.asarray(Ppi.diagonal(), dtype=np.float64)


# --------------------------------------------------------------------------
# Algorithm 1 and the classical methods
# --------------------------------------------------------------------------

@dataclasses.dataclass
class SolveResult:
    V: np.ndarray
    pi: np.ndarray
    converged: bool
    outer_iters: int  # number of policy evaluations performed
    inner_iters: list  # inner iterations per evaluation
    residuals: list  # ||r(V_k)||_inf for k = 0, 1, ...


def ipi(S: int, A: int, row_ptr, col, val, g, gamma: float, V0=None, tol: float = 1e-8,
        alpha: float = 1e-4, max_outer: int = 1000, max_inner: int = 1000, inner: str = "gmres",
        restart: int = 30, omega: float = 1.0) -> SolveResult:
    """Inexact policy iteration, Algorithm 1, with a GMRES, TFQMR, Richardson or
    Jacobi-preconditioned Richardson inner solver.

    k = 0, V = V_0.  Repeat: (TV, pi_{k+1}, res_k) = Bellman step at V_k (steps
    2-3); stop if res_k <= tol, or after max_outer evaluations; otherwise solve
    J_pi theta = g_pi from theta_0 = V_k until ||g_pi - J_pi theta||_2 <
    alpha res_k or max_inner iterations (steps 4-12, Sec. III-B.3), and set
    V_{k+1} = theta.  Returns V_k and the greedy policy of V_k.
    """
    P = stacked_matrix(S, A, row_ptr, col, val)
    V = np.zeros(S) if V0 is None else np.array(V0, dtype=np.float64, copy=True)
    inner_its, residuals = [], []
    k = 0
    while True:
        TV, pi, res = bellman(P, g, gamma, V, S, A)
        residuals.append(res)
        if res <= tol:
            return SolveResult(V, pi, True, k, inner_its, residuals)
        if k >= max_outer:
            return SolveResult(V, pi, False, k, inner_its, residuals)
        Ppi, gpi = policy_system(P, g, pi, A)
        mv = lambda x, Ppi=Ppi: apply_J(Ppi, gamma, x)
        if inner == "gmres":
            out = gmres(mv, gpi, V, restart, alpha * res, max_inner)
        elif inner == "richardson":
            out = richardson(mv, gpi, V, omega, alpha * res, max_inner)
        elif inner == "tfqmr":
            out = tfqmr(mv, gpi, V, alpha * res, max_inner)
        elif inner == "jacobi":
            out = jacobi_richardson(mv, jacobi_diagonal(Ppi, gamma), gpi, V, omega, alpha * res, max_inner)
        else:
            raise ValueError(inner)
        inner_its.append(out.iters)
        V = out.x
        k += 1


def value_iteration(S: int, A: int, row_ptr, col, val, g, gamma: float, V0=None, tol: float = 1e-8,
                    max_iter: int = 100000) -> SolveResult:
    """Value iteration V <- TV until ||TV - V||_inf <= tol (Table 2, first row)."""
    P = stacked_matrix(S, A, row_ptr, col, val)
    V = np.zeros(S) if V0 is None else np.array(V0, dtype=np.float64, copy=True)
    residuals = []
    for k in range(max_iter + 1):
        TV, pi, res = bellman(P, g, gamma, V, S, A)
        residuals.append(res)
        if res <= tol:
            return SolveResult(V, pi, True, k, [1] * k, residuals)
        if k == max_iter:
            break
        V = TV
    return SolveResult(V, pi, False, max_iter, [1] * max_iter, residuals)


def evaluate_policy(Ppi, gpi, gamma: float, dense_limit: int = 5000) -> np.ndarray:
    """V_pi solving (I - gamma P_pi) V = g_pi (Eq. 2) by a dense LAPACK solve.

    Only systems of up to dense_limit states are solved (ValueError above it):
    the oracle's exact evaluation is the plain definition, nothing iterative.
    """
    S = gpi.size
    if S > dense_limit:
        raise ValueError(f"exact policy evaluation is dense: S = {S} > dense_limit = {dense_limit}")
    J = np.eye(S) - gamma * Ppi.toarray()
    return np.linalg.solve(J, gpi)


def policy_iteration(S: int, A: int, row_ptr, col, val, g, gamma: float, max_iter: int = 1000,
                     dense_limit: int = 5000):
    """Howard policy iteration with exact evaluation (Table 2, PI row).

    pi_0 is greedy for V = 0.  Each step evaluates V_pi exactly and switches
    pi(s) to the lowest minimiser of Q(s, .) only where it improves on
    Q(s, pi(s)) by more than 1e-13 max(|Q(s, pi(s))|, ||V_pi||_inf): a strict
    improvement at the scale of the values, so that the dense solve's rounding,
    which leaves values of exact zero as +-1e-17, never makes tied actions
    alternate.  Stops when no state changes; returns (V*, pi*, list of V_pi per
    step).
    """
    P = stacked_matrix(S, A, row_ptr, col, val)
    _, pi, _ = bellman(P, g, gamma, np.zeros(S), S, A)
    history = []
    for _ in range(max_iter):
        Ppi, gpi = policy_system(P, g, pi, A)
        V = evaluate_policy(Ppi, gpi, gamma, dense_limit)
        history.append(V)
        Q = q_values(P, g, gamma, V, S, A)
        best = Q.argmin(axis=1)
        cur = Q[np.arange(S), pi]
        better = Q[np.arange(S), best] < cur - 1e-13 * np.maximum(np.abs(cur), np.abs(V).max())
        if not np.any(better):
            return V, pi.astype(np.int32), history
        pi = np.where(better, best, pi).astype(np.int32)
    raise RuntimeError("policy iteration did not terminate")


def brute_force(S: int, A: int, row_ptr, col, val, g, gamma: float):
    """Optimal cost by enumerating all A**S policies (Sec. II: |Pi| <= m**n).

    For each policy the cost V_pi solves Eq. 2 with a dense solve built from
    the A x S x S tensor; V* is the componentwise minimum over policies.
    Returns (V*, list of policies whose V_pi equals V* to 1e-12 relative, all V_pi).
    """
    P = dense_tensor(S, A, row_ptr, col, val)
    G = np.asarray(g, dtype=np.float64).reshape(S, A)
    costs = {}
    for pol in itertools.product(range(A), repeat=S):
        Ppi = np.array([P[pol[s], s, :] for s in range(S)])
        gpi = np.array([G[s, pol[s]] for s in range(S)])
        costs[pol] = np.linalg.solve(np.eye(S) - gamma * Ppi, gpi)
    Vstar = np.min(np.stack(list(costs.values())), axis=0)
    scale = max(1.0, float(np.max(np.abs(Vstar))))
    optimal = [p for p, v in costs.items() if np.max(np.abs(v - Vstar)) <= 1e-12 * scale]
    return Vstar, optimal, costs


def bellman_states(states, row_cols, row_vals, row_g, gamma: float, V, A: int):
    """Q, TV and greedy action for selected states from their own rows only.

    row_cols, row_vals: [len(states) * A, k] arrays holding rows s*A + a in
    order; row_g: [len(states) * A].  Written out per Eq. 3 without the
    stacked matrix, for sampled checks on workloads too large to build.
    """
    n = len(states)
    V = np.asarray(V, dtype=np.float64)
    PV = np.sum(np.asarray(row_vals, dtype=np.float64) * V[np.asarray(row_cols)], axis=1)
    Q = np.asarray(row_g, dtype=np.float64).reshape(n, A) + gamma * PV.reshape(n, A)
    return Q, Q.min(axis=1), Q.argmin(axis=1)


def action_gaps(Q: np.ndarray) -> np.ndarray:
    """Action gap per state: the second-smallest Q(s, .) minus the smallest one,
    counting repeated values (an exact tie gives 0); inf when A == 1.  It decides
    where the greedy policy of Eq. 4 is unique beyond a given rounding band."""
    if Q.shape[1] == 1:
        return np.full(Q.shape[0], np.inf)
    part = np.partition(Q, 1, axis=1)
    return part[:, 1] - part[:, 0]
