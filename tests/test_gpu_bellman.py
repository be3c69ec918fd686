"""Parity of the fused Bellman sweep (Eq. 3-4, Algorithm 1 steps 2-3) with the FP64 oracle."""
import numpy as np
import pytest

from mdpgen import MDPData, banded_birth_death, pendulum_grid, random_sparse, random_value_vector
from oracle import mdp_oracle as O
from tests._util import check_policy, q_tolerance, to_device

pytestmark = pytest.mark.gpu


def _ragged(S, A, seed, kmax=40):
    """Rows of random lengths 1..kmax (non-uniform layout path)."""
    rng = np.random.default_rng(seed)
    R = S * A
    lens = rng.integers(1, kmax + 1, size=R)
    lens[rng.integers(0, R, size=max(1, R // 50))] = kmax * 3  # a few long rows
    lens = np.minimum(lens, S)
    row_ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    col = np.empty(row_ptr[-1], dtype=np.int32)
    val = np.empty(row_ptr[-1])
    for r in range(R):
        c = np.sort(rng.choice(S, size=lens[r], replace=False))
        w = rng.random(lens[r]) + 1e-3
        col[row_ptr[r]:row_ptr[r + 1]] = c
        val[row_ptr[r]:row_ptr[r + 1]] = w / w.sum()
    g = rng.random(R) * 3 - 1
    return MDPData(S, A, row_ptr, col, val, g, 0.95, f"ragged({S},{A})")


CASES = [
    ("c1_shape", lambda: random_sparse(1000, 4, 8, 0.9, seed=1)),
    ("ragged_tail_states", lambda: random_sparse(1037, 3, 5, 0.97, seed=2)),
    ("one_action", lambda: random_sparse(777, 1, 6, 0.9, seed=3)),
    ("many_actions", lambda: random_sparse(300, 33, 7, 0.99, seed=4)),
    ("long_rows", lambda: random_sparse(400, 5, 100, 0.9, seed=5)),
    ("k1_deterministic", lambda: random_sparse(2000, 7, 1, 0.8, seed=6)),
    ("single_state", lambda: random_sparse(1, 6, 1, 0.5, seed=7)),
    ("tiny", lambda: random_sparse(3, 2, 2, 0.5, seed=8)),
    ("banded", lambda: banded_birth_death(5000, 20, 16, 0.999)),
    ("pendulum", lambda: pendulum_grid(60, 50, 9, 0.9999, seed=3)),
    ("ragged_rows", lambda: _ragged(500, 6, 9)),
    ("ragged_rows_big_A", lambda: _ragged(90, 300, 10, kmax=12)),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_bellman_parity(name, make):
    import torch
    from paper_2507_22538_gb300 import mdp
    m = make()
    d = to_device(m)
    with mdp.MDP(m.S, m.A, d["row_ptr"], d["col"], d["val"], d["g"]) as M:
        for seed in (1, 2):
            V = random_value_vector(m.S, seed, scale=1.0 / (1 - m.gamma))
            TV, pi, res = M.bellman(m.gamma, torch.from_numpy(V).cuda())
            torch.cuda.synchronize()
            P = O.stacked_matrix(m.S, m.A, m.row_ptr, m.col, m.val)
            Q = O.q_values(P, m.g, m.gamma, V, m.S, m.A)
            TVo, pio, reso = O.bellman(P, m.g, m.gamma, V, m.S, m.A)
            tol = q_tolerance(m, V)
            np.testing.assert_allclose(TV.cpu().numpy(), TVo, rtol=0, atol=tol)
            assert abs(res.item() - reso) <= tol
            check_policy(pi.cpu().numpy(), Q, tol)


def test_host_upload_matches_device_upload():
    import torch
    from paper_2507_22538_gb300 import mdp
    m = random_sparse(700, 5, 9, 0.9, seed=12)
    V = torch.from_numpy(random_value_vector(m.S, 3, 10.0)).cuda()
    with mdp.MDP.from_data(m) as Mh:
        a = Mh.bellman(m.gamma, V)
    d = to_device(m)
    with mdp.MDP(m.S, m.A, d["row_ptr"], d["col"], d["val"], d["g"]) as Md:
        b = Md.bellman(m.gamma, V)
    torch.cuda.synchronize()
    for x, y in zip(a, b):
        assert torch.equal(x, y)  # same layout, same kernel: bitwise equal


def _two_chunk_mdp():
    """A banded MDP of 35.2e6 entries (host uploads go in chunks of at most 2^25 entries,
    so this one takes two, with a chunk boundary inside the band) whose rows have 9 or 8
    entries: every fifth row moves the mass of its last entry onto its first one."""
    from mdpgen import banded_birth_death
    m = banded_birth_death(400000, 10, 4, 0.99, quant_bits=11)
    R = m.S * m.A
    col, val = m.col.reshape(R, 9), m.val.reshape(R, 9).copy()
    short = np.arange(R) % 5 == 0
    val[short, 0] += val[short, 8]  # multiples of 2^-11: exact
    keep = np.ones((R, 9), dtype=bool)
    keep[short, 8] = False
    rp = np.zeros(R + 1, dtype=np.int64)
    rp[1:] = np.cumsum(9 - short.astype(np.int64))
    assert rp[-1] > 2 ** 25
    return m, rp, np.ascontiguousarray(col[keep]), np.ascontiguousarray(val[keep])


def test_chunked_host_upload_matches_device_upload():
    import torch
    from paper_2507_22538_gb300 import mdp
    m, rp, col, val = _two_chunk_mdp()
    V = torch.from_numpy(random_value_vector(m.S, 4, 100.0)).cuda()
    host16 = torch.from_numpy(val).to(torch.float16)
    assert torch.equal(host16.double(), torch.from_numpy(val))
    with mdp.MDP(m.S, m.A, torch.from_numpy(rp).cuda(), torch.from_numpy(col).cuda(), torch.from_numpy(val).cuda(),
                 torch.from_numpy(m.g).cuda()) as Md:
        ref = Md.bellman(m.gamma, V)
        for v in (val, torch.from_numpy(val).pin_memory(), host16.pin_memory()):
            with mdp.MDP(m.S, m.A, rp, col, v, m.g) as Mh:
                got = Mh.bellman(m.gamma, V)
                torch.cuda.synchronize()
                for x, y in zip(ref, got):
                    assert torch.equal(x, y)


@pytest.mark.parametrize("bad", ["negative_last", "column_last", "row_sum_first"])
def test_chunked_host_upload_rejects_invalid_entries(bad):
    from paper_2507_22538_gb300 import mdp
    m, rp, col, val = _two_chunk_mdp()
    if bad == "negative_last":  # an entry of the second chunk
        val[-2] = -val[-2]
    elif bad == "column_last":
        col[-1] = m.S
    else:
        val[0] *= 1.5
    st, h = mdp.mdp_create(m.S, m.A, rp, col, val, m.g, False, stream=0)
    assert st == mdp.MDP_ERR_NOT_STOCHASTIC, (st, mdp.mdp_last_error())
    assert not h.value


def test_exact_ties_take_lowest_action():
    """g = 1/4 everywhere, gamma = 3/4, dyadic probabilities, V = 1: every Q is exactly 1."""
    import torch
    from paper_2507_22538_gb300 import mdp
    m = random_sparse(1000, 9, 6, 0.75, seed=4, quant_bits=11)
    with mdp.MDP(m.S, m.A, m.row_ptr, m.col, m.val, np.full_like(m.g, 0.25)) as M:
        TV, pi, res = M.bellman(0.75, torch.ones(m.S, dtype=torch.float64, device="cuda"))
        torch.cuda.synchronize()
        assert torch.all(TV == 1.0) and torch.all(pi == 0) and res.item() == 0.0


def test_nan_input_gives_nan_residual():
    import torch
    from paper_2507_22538_gb300 import mdp
    m = random_sparse(500, 4, 8, 0.9, seed=1)
    with mdp.MDP.from_data(m) as M:
        V = torch.zeros(m.S, dtype=torch.float64, device="cuda")
        V[123] = float("nan")
        TV, pi, res = M.bellman(0.9, V)
        torch.cuda.synchronize()
        assert torch.isnan(res).item()


def test_deterministic_repeat():
    import torch
    from paper_2507_22538_gb300 import mdp
    m = banded_birth_death(3000, 20, 16, 0.999)
    with mdp.MDP.from_data(m) as M:
        V = torch.from_numpy(random_value_vector(m.S, 5, 100.0)).cuda()
        a = M.bellman(m.gamma, V)
        b = M.bellman(m.gamma, V)
        torch.cuda.synchronize()
        for x, y in zip(a, b):
            assert torch.equal(x, y)


@pytest.mark.parametrize("bad", ["row_sum", "column", "negative", "empty_row", "nan_cost", "row_ptr_start", "gamma"])
def test_invalid_inputs_are_rejected(bad):
    import torch
    from paper_2507_22538_gb300 import mdp
    m = random_sparse(50, 3, 4, 0.9, seed=2)
    rp, col, val, g = m.row_ptr.copy(), m.col.copy(), m.val.copy(), m.g.copy()
    expect = mdp.MDP_ERR_NOT_STOCHASTIC
    if bad == "row_sum":
        val[5] *= 1.01
    elif bad == "column":
        col[7] = 50
    elif bad == "negative":
        val[3] = -val[3]
    elif bad == "empty_row":
        rp[1] = 0  # row 0 empty (row 1 then holds two rows' entries)
    elif bad == "nan_cost":
        g[4] = np.nan
        expect = mdp.MDP_ERR_INVALID_ARG
    elif bad == "row_ptr_start":  # one unused entry in front: row_ptr[0] = 1, otherwise a valid CSR
        rp = rp + 1
        rp[0] = 1
        col, val = np.concatenate([[0], col]).astype(np.int32), np.concatenate([[1.0], val])
        expect = mdp.MDP_ERR_INVALID_ARG
    if bad == "gamma":
        with mdp.MDP(m.S, m.A, rp, col, val, g) as M:
            V = torch.zeros(m.S, dtype=torch.float64, device="cuda")
            TV = torch.empty_like(V)
            pi = torch.empty(m.S, dtype=torch.int32, device="cuda")
            assert mdp.mdp_bellman(M.h, 1.0, V, TV, pi) == mdp.MDP_ERR_INVALID_ARG
            assert mdp.mdp_bellman(M.h, 0.9, V, V, pi) == mdp.MDP_ERR_INVALID_ARG
        return
    st, h = mdp.mdp_create(m.S, m.A, rp, col, val, g, False, stream=0)
    assert st == expect, (st, mdp.mdp_last_error())
    assert not h.value


@pytest.mark.parametrize("S,A,k", [(3000, 32, 12), (5000, 3, 7), (700, 100, 5)])
def test_tune_keeps_results(S, A, k):
    """mdp_tune picks a tile size by timing; the Bellman outputs stay bit for bit the same."""
    import torch
    from mdpgen import random_sparse, random_value_vector
    from paper_2507_22538_gb300 import mdp
    m = random_sparse(S, A, k, 0.95, seed=4)
    V = torch.from_numpy(random_value_vector(S, 2, 5.0)).cuda()
    with mdp.MDP.from_data(m) as M:
        TV0, pi0, r0 = M.bellman(m.gamma, V)
        st, ts, ms = mdp.mdp_tune(M.h, m.gamma)
        assert st == mdp.MDP_OK and ts in (8, 16, 32, 64, 128, 256, 512) and ms > 0
        TV1, pi1, r1 = M.bellman(m.gamma, V)
        torch.cuda.synchronize()
    assert torch.equal(TV0, TV1) and torch.equal(pi0, pi1) and torch.equal(r0, r1)


SHAPES = [(tile, rpw, vb, bps) for tile in (8, 37, 64, 256) for rpw in (32, 64) for vb in (16, 32)
          for bps in (0, 1)]


@pytest.mark.parametrize("name", ["c1_shape", "ragged_tail_states", "many_actions", "long_rows", "k1_deterministic",
                                  "tiny", "banded", "ragged_rows", "ragged_rows_big_A"])
def test_every_sweep_shape_gives_the_same_bits(name):
    """The launch shapes the tuner chooses among (states per tile, 32 or 64 rows per
    warp step, 16- or 32-byte value loads, blocks per SM): every one gives the oracle-
    checked default sweep's TV, policy and residual bit for bit."""
    import torch
    from paper_2507_22538_gb300 import mdp
    m = dict(CASES)[name]()
    V = torch.from_numpy(random_value_vector(m.S, 3, scale=1.0 / (1 - m.gamma))).cuda()
    with mdp.MDP.from_data(m) as M:
        TV0, pi0, r0 = M.bellman(m.gamma, V)
        seen = 0
        for tile, rpw, vb, bps in SHAPES:
            st = mdp.mdp_set_sweep_shape(M.h, tile, rpw, vb, bps)
            if tile * m.A * 8 > 227 * 1024:
                assert st == mdp.MDP_ERR_INVALID_ARG
                continue
            assert st == mdp.MDP_OK, mdp.mdp_last_error()
            st, shape = mdp.mdp_get_sweep_shape(M.h)
            assert shape["tile_states"] == tile and shape["rows_per_warp"] == rpw
            assert shape["value_load_bytes"] == vb and shape["blocks"] >= 1
            TV1, pi1, r1 = M.bellman(m.gamma, V)
            torch.cuda.synchronize()
            assert torch.equal(TV0, TV1) and torch.equal(pi0, pi1) and torch.equal(r0, r1), (tile, rpw, vb, bps)
            seen += 1
        assert seen >= 8
        assert mdp.mdp_set_sweep_shape(M.h, 64, 48, 16, 0) == mdp.MDP_ERR_INVALID_ARG
        assert mdp.mdp_set_sweep_shape(M.h, 64, 32, 8, 0) == mdp.MDP_ERR_INVALID_ARG
        assert mdp.mdp_set_sweep_shape(M.h, 0, 32, 16, 0) == mdp.MDP_ERR_INVALID_ARG


def test_tuned_shape_solves_the_same():
    """After mdp_tune (tile, rows per warp step, load width, grid) a stream- and a
    graph-driven solve give the untuned solve's V, policy and counts bit for bit."""
    import torch
    from paper_2507_22538_gb300 import mdp
    m = banded_birth_death(20000, 20, 33, 0.999)
    with mdp.MDP.from_data(m) as M:
        def solve(graph):
            V = torch.zeros(m.S, dtype=torch.float64, device="cuda")
            pi = torch.empty(m.S, dtype=torch.int32, device="cuda")
            o = mdp.mdp_default_opts()
            o.gamma, o.atol_pi, o.alpha, o.graph = m.gamma, 1e-8, 0.01, graph
            st, stats = mdp.mdp_solve(M.h, o, V, pi, None)
            torch.cuda.synchronize()
            assert st == mdp.MDP_OK
            return V.cpu(), pi.cpu(), stats.outer_iters, stats.inner_iters_total, stats.final_residual
        ref = solve(0)
        st, ts, ms = mdp.mdp_tune(M.h, m.gamma)
        assert st == mdp.MDP_OK
        st, shape = mdp.mdp_get_sweep_shape(M.h)
        assert shape["rows_per_warp"] in (32, 64) and shape["value_load_bytes"] in (16, 32)
        for graph in (0, 1):
            out = solve(graph)
            assert torch.equal(out[0], ref[0]) and torch.equal(out[1], ref[1]) and out[2:] == ref[2:]
        # a hand-set shape of each variant
        for rpw, vb in ((64, 32), (32, 32), (64, 16)):
            assert mdp.mdp_set_sweep_shape(M.h, 32, rpw, vb, 0) == mdp.MDP_OK
            out = solve(1)
            assert torch.equal(out[0], ref[0]) and torch.equal(out[1], ref[1]) and out[2:] == ref[2:]


def test_live_handle_survives_a_handle_with_a_smaller_tile():
    """The sweep's dynamic shared memory cap is one setting per kernel and device,
    shared by all handles: creating a handle whose Q tile needs less (A = 29: 256
    states x 29 actions x 8 B = 59 KB) must not lower it under a live handle whose
    tile needs more (A = 31: 63.5 KB), whose sweeps would then be refused.  Requests
    of different A solved concurrently by the serving loop meet exactly this."""
    import torch
    from paper_2507_22538_gb300 import mdp
    mx = random_sparse(600, 31, 4, 0.9, seed=21)
    my = random_sparse(600, 29, 4, 0.9, seed=22)
    with mdp.MDP.from_data(mx) as X, mdp.MDP.from_data(my) as Y:
        for M, m in ((X, mx), (Y, my), (X, mx)):
            V = random_value_vector(m.S, 1, scale=1.0 / (1 - m.gamma))
            TV, pi, res = M.bellman(m.gamma, torch.from_numpy(V).cuda())
            torch.cuda.synchronize()
            P = O.stacked_matrix(m.S, m.A, m.row_ptr, m.col, m.val)
            TVo, _, reso = O.bellman(P, m.g, m.gamma, V, m.S, m.A)
            tol = q_tolerance(m, V)
            np.testing.assert_allclose(TV.cpu().numpy(), TVo, rtol=0, atol=tol)
            assert abs(res.item() - reso) <= tol
