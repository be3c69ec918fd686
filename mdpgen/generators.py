"""Seeded synthetic MDP generators (inputs only; no MDP solution arithmetic).

Every generator returns an ``MDPData``: the row-stacked transition matrix of
Eq. 5 in CSR form (row index s*A + a holds P(s, ., a)) and the stage costs g
as an S x A row-major array (g[s*A + a] = g(s, a)), plus the discount factor.

Random draws come from Philox4x32-10 keyed by (seed, stream tag) with the
counter set to (global row index, draw index), so any row can be regenerated
alone (see ``regenerate_rows``).  The workloads mirror the shapes used in the
paper's experiments (Sec. IV): random sparse MDPs with uniform columns
(Sec. IV-A), a banded birth-death chain standing in for the SIS epidemic model
(Sec. IV-B), a bilinear-interpolated pendulum grid (Sec. IV-C) and a
deterministic maze (Sec. IV-D).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from .philox import stream

# stream tags: one Philox key word per purpose so that draws never overlap
TAG_COLS = 0x636F6C73  # "cols"
TAG_VALS = 0x76616C73  # "vals"
TAG_COST = 0x636F7374  # "cost"
TAG_NOISE = 0x6E6F6973  # "nois"


@dataclasses.dataclass
class MDPData:
    S: int
    A: int
    row_ptr: np.ndarray  # int64 [S*A + 1]
    col: np.ndarray  # int32 [nnz]
    val: np.ndarray  # float64 [nnz]
    g: np.ndarray  # float64 [S*A]
    gamma: float
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def row(self, s: int, a: int):
        r = s * self.A + a
        lo, hi = int(self.row_ptr[r]), int(self.row_ptr[r + 1])
        return self.col[lo:hi], self.val[lo:hi]


# --------------------------------------------------------------------------
# value transforms
# --------------------------------------------------------------------------

def quantize_rows(w: np.ndarray, bits: int) -> np.ndarray:
    """Round each row of nonnegative weights to multiples of 2**-bits summing to 1.

    Largest-remainder rounding: each row is scaled to 2**bits units, floored,
    and the missing units go to the entries with the largest remainders (ties
    to the lower position).  The result is exactly representable in binary16
    for bits <= 11 and in bfloat16 for bits <= 8, and every row sums to
    exactly one in binary64.
    """
    unit = float(1 << bits)
    w = np.asarray(w, dtype=np.float64)
    x = w / w.sum(axis=1, keepdims=True) * unit
    q = np.floor(x)
    missing = (unit - q.sum(axis=1)).astype(np.int64)
    rem = x - q
    # stable order: larger remainder first, then lower position first
    order = np.argsort(-rem, axis=1, kind="stable")
    ranks = np.empty_like(order)
    np.put_along_axis(ranks, order, np.arange(w.shape[1])[None, :].repeat(w.shape[0], 0), axis=1)
    q += (ranks < missing[:, None]).astype(np.float64)
    return q / unit


def _dirichlet_weights(seed: int, rows: np.ndarray, k: int, conc: float) -> np.ndarray:
    """Unnormalised Dirichlet(conc) weights for k entries of each given row.

    conc == 1: Gamma(1) = -log(U) (exponential).
    conc == 0.5: Gamma(1/2) = Z**2 / 2 with Z standard normal (Box-Muller).
    """
    j = np.arange(k, dtype=np.uint64)[None, :]
    r = rows.astype(np.uint64)[:, None]
    if conc == 1.0:
        u = stream(seed, TAG_VALS, r, j)
        return -np.log1p(-u)  # U in [0,1) -> 1-U in (0,1]
    if conc == 0.5:
        u1 = stream(seed, TAG_VALS, r, j, lane=0)
        u2 = stream(seed, TAG_VALS, r, j, lane=1)
        z = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)
        w = 0.5 * z * z
        # a row of all-zero weights cannot be normalised: give it uniform mass
        dead = w.sum(axis=1) <= 0.0
        if np.any(dead):
            w[dead] = 1.0
        return w
    raise ValueError("supported Dirichlet concentrations: 1.0, 0.5")


def _distinct_columns(seed: int, rows: np.ndarray, k: int, S: int) -> np.ndarray:
    """k distinct uniform columns in [0, S) per row, sorted ascending (Floyd's algorithm)."""
    if k > S:
        raise ValueError("k > S")
    n = rows.shape[0]
    chosen = np.empty((n, k), dtype=np.int64)
    r = rows.astype(np.uint64)
    for i in range(k):
        jmax = S - k + i  # draw t uniformly in [0, jmax]
        u = stream(seed, TAG_COLS, r, np.uint64(i))
        t = np.minimum(np.floor(u * (jmax + 1)).astype(np.int64), jmax)
        if i:
            dup = (chosen[:, :i] == t[:, None]).any(axis=1)
            t = np.where(dup, jmax, t)
        chosen[:, i] = t
    chosen.sort(axis=1)
    return chosen


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def random_sparse(S: int, A: int, k: int, gamma: float, seed: int, conc: float = 1.0,
                  quant_bits: int | None = None, chunk_rows: int = 1 << 20) -> MDPData:
    """Random sparse MDP in the style of Sec. IV-A.

    Each (s, a) row has k distinct columns drawn uniformly, probabilities
    Dirichlet(conc) (optionally quantised to 2**-quant_bits, explicit zeros
    kept so every row has exactly k entries), and costs g(s, a) ~ U[0, 1).
    """
    R = S * A
    col = np.empty(R * k, dtype=np.int32)
    val = np.empty(R * k, dtype=np.float64)
    for r0 in range(0, R, chunk_rows):
        r1 = min(R, r0 + chunk_rows)
        rows = np.arange(r0, r1, dtype=np.int64)
        c = _distinct_columns(seed, rows, k, S)
        w = _dirichlet_weights(seed, rows, k, conc)
        if quant_bits is None:
            p = w / w.sum(axis=1, keepdims=True)
        else:
            p = quantize_rows(w, quant_bits)
        col[r0 * k:r1 * k] = c.ravel()
        val[r0 * k:r1 * k] = p.ravel()
    g = stream(seed, TAG_COST, np.arange(R, dtype=np.uint64), np.uint64(0))
    row_ptr = np.arange(R + 1, dtype=np.int64) * k
    return MDPData(S, A, row_ptr, col, val, g, gamma, f"random_sparse(S={S},A={A},k={k})")


def ragged_sparse(S: int, A: int, kmax: int, gamma: float, seed: int, long_frac: float = 0.02,
                  quant_bits: int | None = None) -> MDPData:
    """Random sparse MDP whose rows have different lengths: 1..kmax distinct uniform
    columns (sorted), plus a fraction long_frac of rows with 3 kmax entries (capped
    at S), Dirichlet(1) weights (optionally quantised to 2**-quant_bits), costs
    U[-1, 2).  Every row of the stacked matrix and of any policy's rows has its own
    length, which exercises the non-uniform sliced layouts.  Drawn with numpy's
    PCG64 from `seed` (test inputs; rows are not regenerated one by one)."""
    rng = np.random.default_rng(seed)
    R = S * A
    lens = rng.integers(1, kmax + 1, size=R)
    lens[rng.integers(0, R, size=max(1, int(R * long_frac)))] = 3 * kmax
    lens = np.minimum(lens, S)
    row_ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    col = np.empty(int(row_ptr[-1]), dtype=np.int32)
    val = np.empty(int(row_ptr[-1]))
    for r in range(R):
        lo, hi = int(row_ptr[r]), int(row_ptr[r + 1])
        col[lo:hi] = np.sort(rng.choice(S, size=hi - lo, replace=False))
        w = -np.log1p(-rng.random(hi - lo))
        val[lo:hi] = w / w.sum() if quant_bits is None else quantize_rows(w[None, :], quant_bits)[0]
    g = rng.random(R) * 3.0 - 1.0
    return MDPData(S, A, row_ptr, col, val, g, gamma, f"ragged_sparse({S},{A},{kmax})")


def sis_band_centres(s: np.ndarray, a: np.ndarray, S: int, A: int, half_width: int,
                     r0_max: float = 2.5) -> np.ndarray:
    """Band centre of row (s, a): the expected infected count after one SIS step.

    As in the SIS model of Sec. IV-B the infectious period is one step, so the
    next infected count is the number of new infections among the S-1-s
    susceptibles, each infected with probability q = 1 - exp(-R0(a) s / S);
    intervention level a scales the reproduction number R0(a) = r0_max (1 - a/A).
    The centre is that mean, rounded and clamped so the band stays in [0, S).
    """
    s = np.asarray(s, dtype=np.float64)
    r0 = r0_max * (1.0 - np.asarray(a, dtype=np.float64) / A)
    mean = (S - 1 - s) * (1.0 - np.exp(-r0 * s / S))
    return np.clip(np.rint(mean), half_width, S - 1 - half_width).astype(np.int64)


def banded_birth_death(S: int = 1_000_000, A: int = 20, half_width: int = 16, gamma: float = 0.999,
                       quant_bits: int | None = None, chunk_states: int = 1 << 16) -> MDPData:
    """Banded epidemic-like MDP standing in for the SIS model of Sec. IV-B.

    State s is the infected count, action a an intervention level.  Row (s, a)
    is a band of 2h+1 contiguous columns centred at ``sis_band_centres`` (the
    expected infected count one step later) holding the Binomial(2h, 1/2) pmf
    C(2h, j) / 2**(2h), exact in binary64 (or, with quant_bits, rounded to
    2**-quant_bits by largest remainder).  Cost g(s, a) = s/S + 0.05 a.
    """
    h = half_width
    w = 2 * h + 1
    if S < w:
        raise ValueError("S must be at least the band width")
    pmf = np.array([math.comb(2 * h, j) for j in range(w)], dtype=np.float64) / float(2 ** (2 * h))
    if quant_bits is not None:
        pmf = quantize_rows(pmf[None, :], quant_bits)[0]
    R = S * A
    col = np.empty(R * w, dtype=np.int32)
    val = np.empty(R * w, dtype=np.float64)
    offs = np.arange(-h, h + 1, dtype=np.int64)
    acts = np.arange(A, dtype=np.int64)
    for s0 in range(0, S, chunk_states):
        s1 = min(S, s0 + chunk_states)
        s = np.arange(s0, s1, dtype=np.int64)
        c = sis_band_centres(s[:, None], acts[None, :], S, A, h)  # [ns, A]
        cols = c[:, :, None] + offs[None, None, :]
        lo, hi = s0 * A * w, s1 * A * w
        col[lo:hi] = cols.ravel()
        val[lo:hi] = np.broadcast_to(pmf, cols.shape).ravel()
    s_all = np.repeat(np.arange(S, dtype=np.float64), A)
    a_all = np.tile(np.arange(A, dtype=np.float64), S)
    g = s_all / S + 0.05 * a_all
    row_ptr = np.arange(R + 1, dtype=np.int64) * w
    return MDPData(S, A, row_ptr, col, val, g, gamma, f"banded_birth_death(S={S},A={A},k={w})")


def pendulum_grid(n_theta: int = 1000, n_omega: int = 1000, A: int = 9, gamma: float = 0.9999,
                  seed: int = 3, Ts: float = 0.01, quant_bits: int | None = None,
                  chunk_states: int = 1 << 16) -> MDPData:
    """Inverted-pendulum grid MDP after Sec. IV-C (Eq. 8-10).

    State s = i_theta * n_omega + i_omega on theta in [0, 2 pi) (periodic, step
    2 pi / n_theta) and omega on linspace(-10, 10, n_omega); torques F on
    linspace(-3, 3, A).  One forward-Euler step (theta' = theta + Ts omega,
    omega' = omega + Ts (F - 9.80665 sin theta)) plus a Gaussian offset with
    standard deviation half a grid step per dimension (drawn once per (s, a))
    gives a continuous successor that is spread over its 4 surrounding grid
    nodes by bilinear weights (omega clamped inside the grid so the 4 nodes are
    distinct).  Cost g = 2 [(theta - pi)^2 + omega^2] + F^2.
    """
    S = n_theta * n_omega
    R = S * A
    dth = 2.0 * math.pi / n_theta
    om = np.linspace(-10.0, 10.0, n_omega)
    dom = om[1] - om[0]
    forces = np.linspace(-3.0, 3.0, A)
    col = np.empty(R * 4, dtype=np.int32)
    val = np.empty(R * 4, dtype=np.float64)
    g = np.empty(R, dtype=np.float64)
    for s0 in range(0, S, chunk_states):
        s1 = min(S, s0 + chunk_states)
        s = np.arange(s0, s1, dtype=np.int64)
        ith, iom = s // n_omega, s % n_omega
        th = ith * dth
        w_ = om[iom]
        rows = (s[:, None] * A + np.arange(A)[None, :]).astype(np.uint64)  # [ns, A]
        F = forces[None, :]
        thn = th[:, None] + Ts * w_[:, None]
        omn = w_[:, None] + Ts * (F - 9.80665 * np.sin(th)[:, None])
        # Gaussian offsets via Box-Muller from one Philox block per row
        u1 = stream(seed, TAG_NOISE, rows, np.uint64(0), lane=0)
        u2 = stream(seed, TAG_NOISE, rows, np.uint64(0), lane=1)
        rad = np.sqrt(-2.0 * np.log1p(-u1))
        z1 = rad * np.cos(2.0 * math.pi * u2)
        z2 = rad * np.sin(2.0 * math.pi * u2)
        thn = thn + 0.5 * dth * z1
        omn = omn + 0.5 * dom * z2
        # theta: periodic cell index and fraction
        xt = np.mod(thn, 2.0 * math.pi) / dth
        i0 = np.floor(xt).astype(np.int64)
        ft = xt - i0
        i0 = np.mod(i0, n_theta)
        i1 = np.mod(i0 + 1, n_theta)
        # omega: clamp inside the grid
        xo = np.clip((omn - om[0]) / dom, 0.0, n_omega - 1.0)
        j0 = np.minimum(np.floor(xo).astype(np.int64), n_omega - 2)
        fo = xo - j0
        j1 = j0 + 1
        cols = np.stack([i0 * n_omega + j0, i0 * n_omega + j1, i1 * n_omega + j0, i1 * n_omega + j1], axis=-1)
        wts = np.stack([(1 - ft) * (1 - fo), (1 - ft) * fo, ft * (1 - fo), ft * fo], axis=-1)
        order = np.argsort(cols, axis=-1, kind="stable")
        cols = np.take_along_axis(cols, order, axis=-1)
        wts = np.take_along_axis(wts, order, axis=-1)
        wts = wts.reshape(-1, 4)
        if quant_bits is not None:
            wts = quantize_rows(wts, quant_bits)
        else:
            wts = wts / wts.sum(axis=1, keepdims=True)
        lo, hi = s0 * A * 4, s1 * A * 4
        col[lo:hi] = cols.ravel()
        val[lo:hi] = wts.ravel()
        gg = 2.0 * ((th[:, None] - math.pi) ** 2 + w_[:, None] ** 2) + F ** 2
        g[s0 * A:s1 * A] = gg.ravel()
    row_ptr = np.arange(R + 1, dtype=np.int64) * 4
    return MDPData(S, A, row_ptr, col, val, g, gamma, f"pendulum_grid({n_theta}x{n_omega},A={A})")


def maze(H: int, W: int, wall_frac: float = 0.2, seed: int = 7, gamma: float = 0.99,
         goal_cost: float = -100.0, bump_cost: float = 1.0) -> tuple[MDPData, np.ndarray, int]:
    """Deterministic grid maze after Sec. IV-D, with walls removed from the state space.

    Cells are drawn as walls with probability wall_frac (the goal, the
    bottom-right cell, is always free).  States are the free cells in
    row-major order.  Actions 0..4 = stay, north, east, south, west.  A move
    into a wall or off the grid leaves the agent in place at cost bump_cost;
    other moves cost 0, and every action taken in the goal keeps the agent
    there at cost goal_cost.  Returns (mdp, free-cell grid index of each
    state, goal state index).
    """
    u = stream(seed, TAG_COLS, np.arange(H * W, dtype=np.uint64), np.uint64(0)).reshape(H, W)
    wall = u < wall_frac
    wall[H - 1, W - 1] = False
    free_idx = np.flatnonzero(~wall.ravel())
    state_of = -np.ones(H * W, dtype=np.int64)
    state_of[free_idx] = np.arange(free_idx.size)
    S, A = free_idx.size, 5
    goal = int(state_of[(H - 1) * W + (W - 1)])
    moves = [(0, 0), (-1, 0), (0, 1), (1, 0), (0, -1)]
    col = np.empty(S * A, dtype=np.int32)
    g = np.zeros(S * A, dtype=np.float64)
    ys, xs = free_idx // W, free_idx % W
    for a, (dy, dx) in enumerate(moves):
        ny, nx = ys + dy, xs + dx
        inside = (ny >= 0) & (ny < H) & (nx >= 0) & (nx < W)
        tgt = np.where(inside, ny * W + nx, 0)
        ok = inside & ~wall.ravel()[tgt]
        nxt = np.where(ok, state_of[tgt], np.arange(S))
        cost = np.where(ok | (a == 0), 0.0, bump_cost)
        nxt[goal] = goal
        cost[goal] = goal_cost
        col[np.arange(S) * A + a] = nxt
        g[np.arange(S) * A + a] = cost
    val = np.ones(S * A, dtype=np.float64)
    row_ptr = np.arange(S * A + 1, dtype=np.int64)
    return MDPData(S, A, row_ptr, col, val, g, gamma, f"maze({H}x{W})"), free_idx, goal


def serving_request(rid: int, seed: int = 5, s_range=(1_000, 1_000_000), a_range=(2, 32), k_range=(4, 64),
                    gammas=(0.9, 0.99, 0.999, 0.9999)) -> MDPData:
    """One request of a serving stream: S log-uniform in s_range, A and k uniform in
    their ranges (k fixed over the request's rows), gamma drawn from `gammas`,
    k uniform columns per row (drawn with replacement, sorted; a repeated column
    simply adds its probabilities), Dirichlet(1) probabilities, costs U[0, 1).
    Drawn from numpy's PCG64 seeded with (seed, rid), so any request is reproducible
    alone."""
    rng = np.random.Generator(np.random.PCG64([seed, rid]))
    lo, hi = math.log(s_range[0]), math.log(s_range[1])
    S = int(round(math.exp(rng.uniform(lo, hi))))
    A = int(rng.integers(a_range[0], a_range[1] + 1))
    k = int(min(S, rng.integers(k_range[0], k_range[1] + 1)))
    gamma = float(gammas[int(rng.integers(0, len(gammas)))])
    R = S * A
    col = np.sort(rng.integers(0, S, size=(R, k), dtype=np.int32), axis=1).ravel()
    w = rng.exponential(1.0, size=(R, k)) + 1e-12
    val = (w / w.sum(axis=1, keepdims=True)).ravel()
    g = rng.random(R)
    row_ptr = np.arange(R + 1, dtype=np.int64) * k
    return MDPData(S, A, row_ptr, col, val, g, gamma, f"request{rid}(S={S},A={A},k={k},gamma={gamma})")


TAG_REQ = 0x72657173  # "reqs"
REQUEST_ROW_BITS = 40  # request rid's rows use Philox row counters rid * 2**40 + r


def request_header(rid: int, seed: int, s_range=(1_000, 1_000_000), a_range=(2, 32), k_range=(4, 64),
                   gammas=(0.9, 0.99, 0.999, 0.9999)):
    """(S, A, k, gamma) of request rid of the counter-based serving stream: S
    log-uniform in s_range, A and k uniform in their ranges (k <= S), gamma drawn
    from `gammas`; four Philox draws at counter (rid, 0..3)."""
    u = stream(seed, TAG_REQ, np.uint64(rid), np.arange(4, dtype=np.uint64))
    lo, hi = math.log(s_range[0]), math.log(s_range[1])
    S = int(round(math.exp(lo + float(u[0]) * (hi - lo))))
    A = a_range[0] + min(int(float(u[1]) * (a_range[1] - a_range[0] + 1)), a_range[1] - a_range[0])
    k = min(S, k_range[0] + min(int(float(u[2]) * (k_range[1] - k_range[0] + 1)), k_range[1] - k_range[0]))
    gamma = float(gammas[min(int(float(u[3]) * len(gammas)), len(gammas) - 1)])
    return S, A, k, gamma


def serving_request_philox(rid: int, seed: int = 5, s_range=(1_000, 1_000_000), a_range=(2, 32),
                           k_range=(4, 64), gammas=(0.9, 0.99, 0.999, 0.9999)) -> MDPData:
    """Request rid of the counter-based serving stream (the header of
    request_header).  Row r of the request draws from Philox row counter
    rid * 2**40 + r: k uniform columns with replacement (draw j at block j,
    sorted; a repeated column adds its probabilities), Dirichlet(1) weights
    -log(1 - U) (block k + j), normalised, and a cost U[0, 1) (stream TAG_COST).
    Any request, or any row of it, is reproducible alone, and
    mdpgen.torch_gen.serving_request_device draws the same request on the
    device."""
    S, A, k, gamma = request_header(rid, seed, s_range, a_range, k_range, gammas)
    R = S * A
    rows = (np.uint64(rid) << np.uint64(REQUEST_ROW_BITS)) + np.arange(R, dtype=np.uint64)
    j = np.arange(k, dtype=np.uint64)[None, :]
    u = stream(seed, TAG_COLS, rows[:, None], j)
    col = np.minimum(np.floor(u * S).astype(np.int64), S - 1)
    col.sort(axis=1)
    w = -np.log1p(-stream(seed, TAG_VALS, rows[:, None], j + np.uint64(k)))
    val = w / w.sum(axis=1, keepdims=True)
    g = stream(seed, TAG_COST, rows, np.uint64(0))
    row_ptr = np.arange(R + 1, dtype=np.int64) * k
    return MDPData(S, A, row_ptr, col.astype(np.int32).ravel(), val.ravel(), g, gamma,
                   f"request{rid}(S={S},A={A},k={k},gamma={gamma})")


def random_value_vector(S: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """A seeded test vector V ~ scale * U[-1, 1) of length S."""
    u = stream(seed, TAG_NOISE ^ 0x5A5A, np.arange(S, dtype=np.uint64), np.uint64(1))
    return scale * (2.0 * u - 1.0)


def regenerate_rows(kind: str, params: dict, rows: np.ndarray):
    """Regenerate selected CSR rows of a workload without building the whole matrix.

    Returns (cols [n, k] int64, vals [n, k] float64, g [n]) for the given
    global row indices.  Supported kinds: "random_sparse", "banded_birth_death".
    """
    rows = np.asarray(rows, dtype=np.int64)
    if kind == "random_sparse":
        S, A, k, seed = params["S"], params["A"], params["k"], params["seed"]
        conc, qb = params.get("conc", 1.0), params.get("quant_bits")
        c = _distinct_columns(seed, rows, k, S)
        w = _dirichlet_weights(seed, rows, k, conc)
        p = w / w.sum(axis=1, keepdims=True) if qb is None else quantize_rows(w, qb)
        g = stream(seed, TAG_COST, rows.astype(np.uint64), np.uint64(0))
        return c, p, g
    if kind == "banded_birth_death":
        S, A = params["S"], params["A"]
        h = params.get("half_width", 16)
        qb = params.get("quant_bits")
        w = 2 * h + 1
        pmf = np.array([math.comb(2 * h, j) for j in range(w)], dtype=np.float64) / float(2 ** (2 * h))
        if qb is not None:
            pmf = quantize_rows(pmf[None, :], qb)[0]
        s, a = rows // A, rows % A
        c = sis_band_centres(s, a, S, A, h)
        cols = c[:, None] + np.arange(-h, h + 1)[None, :]
        return cols, np.broadcast_to(pmf, cols.shape).copy(), s / S + 0.05 * a
    raise ValueError(kind)


# named workloads (the shapes of the five benchmark configurations)
def workload(name: str) -> MDPData:
    if name == "random_s1000_a4_k8":
        return random_sparse(1000, 4, 8, 0.9, seed=1, conc=1.0)
    if name == "banded_s1e6_a20_k33":
        return banded_birth_death(1_000_000, 20, 16, 0.999)
    if name == "pendulum_1000x1000_a9":
        return pendulum_grid(1000, 1000, 9, 0.9999, seed=3)
    raise ValueError(name)
