"""Input generators: Philox known answers, row layout (Eq. 5), stochasticity, quantisation."""
import math

import numpy as np
import pytest

from mdpgen import (banded_birth_death, pendulum_grid, philox4x32, quantize_rows, random_sparse,
                    regenerate_rows)


def test_philox_known_answers():
    """Philox4x32-10 known-answer vectors published with the Random123 library."""
    cases = [
        ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
        ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
        ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
         (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
    ]
    for ctr, key, expect in cases:
        assert tuple(int(x) for x in philox4x32(ctr, key)) == expect


def _row_sums(m):
    return np.add.reduceat(m.val, m.row_ptr[:-1])


def test_random_sparse_shape_and_stochastic():
    m = random_sparse(500, 4, 8, 0.9, seed=1)
    assert m.row_ptr.shape == (2001,) and m.nnz == 16000
    assert np.all(np.diff(m.row_ptr) == 8)
    assert m.col.min() >= 0 and m.col.max() < 500
    cols = m.col.reshape(-1, 8)
    assert np.all(np.diff(cols, axis=1) > 0)  # distinct, ascending
    assert np.all(m.val >= 0)
    assert np.max(np.abs(_row_sums(m) - 1)) < 1e-15
    assert np.all((m.g >= 0) & (m.g < 1))


def test_quantised_rows_sum_exactly_to_one():
    m = random_sparse(300, 3, 32, 0.99, seed=4, conc=0.5, quant_bits=11)
    assert np.all(_row_sums(m) == 1.0)
    assert np.all(m.val * 2048 == np.round(m.val * 2048))
    q = quantize_rows(np.array([[1.0, 1.0, 1.0]]), 8)
    assert q.sum() == 1.0 and sorted((q[0] * 256).tolist()) == [85, 85, 86]


def test_banded_layout_row_is_state_times_A_plus_action():
    """Row s*A + a holds P(s, ., a): the band sits at the expected infected count of
    one SIS step from s under intervention a (Eq. 5 layout)."""
    S, A, h = 200, 6, 4
    m = banded_birth_death(S, A, h, 0.999)
    for s in (0, 57, 199):
        for a in range(A):
            cols, vals = m.row(s, a)
            mean = (S - 1 - s) * (1 - math.exp(-2.5 * (1 - a / A) * s / S))
            c = min(max(int(np.rint(mean)), h), S - 1 - h)
            assert cols.tolist() == list(range(c - h, c + h + 1))
            assert vals.sum() == 1.0
            assert math.isclose(vals[h], math.comb(2 * h, h) / 2 ** (2 * h))
            assert m.g[s * A + a] == s / S + 0.05 * a


def test_pendulum_rows():
    m = pendulum_grid(30, 20, 5, 0.9999, seed=3)
    assert m.S == 600 and m.nnz == 600 * 5 * 4
    assert np.max(np.abs(_row_sums(m) - 1)) < 1e-14
    cols = m.col.reshape(-1, 4)
    assert np.all(np.diff(cols, axis=1) > 0)


def test_regenerate_rows_matches_full_build():
    m = random_sparse(700, 5, 6, 0.9, seed=9)
    rows = np.array([0, 13, 3499])
    c, p, g = regenerate_rows("random_sparse", dict(S=700, A=5, k=6, seed=9), rows)
    for i, r in enumerate(rows):
        lo, hi = m.row_ptr[r], m.row_ptr[r + 1]
        assert np.array_equal(c[i], m.col[lo:hi])
        assert np.array_equal(p[i], m.val[lo:hi])
        assert g[i] == m.g[r]
    b = banded_birth_death(300, 20, 16, 0.999)
    rows = np.array([5, 2000, 5999])
    c, p, g = regenerate_rows("banded_birth_death", dict(S=300, A=20), rows)
    for i, r in enumerate(rows):
        lo, hi = b.row_ptr[r], b.row_ptr[r + 1]
        assert np.array_equal(c[i], b.col[lo:hi]) and np.array_equal(p[i], b.val[lo:hi])
        assert g[i] == b.g[r]


def test_torch_philox_known_answers():
    """The tensor Philox (used to build large workloads on the device) on the same
    Random123 known-answer vectors."""
    import torch

    from mdpgen.torch_gen import philox4x32 as tphilox
    cases = [
        ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
        ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
        ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
         (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
    ]
    for ctr, key, expect in cases:
        out = tphilox(*(torch.tensor([c], dtype=torch.int64) for c in ctr), *key)
        assert tuple(int(x[0]) for x in out) == expect


@pytest.mark.parametrize("conc,quant", [(1.0, None), (0.5, None), (0.5, 11)])
def test_torch_generator_matches_numpy(conc, quant):
    """random_sparse_device (run here on the CPU) against random_sparse: columns, row
    pointers and costs bit for bit; probabilities to rounding, and quantised ones
    equal in all but rare rows, each row summing to exactly 1."""
    import torch

    from mdpgen.torch_gen import random_sparse_device
    m = random_sparse(3000, 5, 16, 0.99, seed=12, conc=conc, quant_bits=quant)
    rp, col, val, g = random_sparse_device(3000, 5, 16, 0.99, seed=12, conc=conc, quant_bits=quant, device="cpu",
                                           chunk_rows=4096)
    assert np.array_equal(rp.numpy(), m.row_ptr)
    assert np.array_equal(col.numpy(), m.col)
    assert np.array_equal(g.numpy(), m.g)
    v = val.numpy().reshape(-1, 16)
    ref = m.val.reshape(-1, 16)
    if quant is None:
        np.testing.assert_allclose(v, ref, rtol=1e-13, atol=1e-16)
    else:
        same = np.all(v == ref, axis=1)
        assert same.mean() > 0.999
        assert np.all(v.sum(axis=1) == 1.0)
        assert np.all(v * 2048 == np.floor(v * 2048))


def test_serving_request_philox_device_matches_numpy():
    """The counter-based serving request drawn with tensor ops (here on the CPU)
    against the numpy draw: header, columns and costs bit for bit, probabilities
    to rounding; every row sums to 1 and columns lie in [0, S)."""
    from mdpgen import request_header, serving_request_philox
    from mdpgen.torch_gen import serving_request_device
    rng = dict(s_range=(200, 3000), a_range=(2, 6), k_range=(3, 9))
    for rid in (0, 1, 7, 123456):
        m = serving_request_philox(rid, seed=3, **rng)
        S, A, k, gamma, rp, col, val, g = serving_request_device(rid, seed=3, device="cpu", chunk_rows=1000, **rng)
        assert (S, A, k, gamma) == (m.S, m.A, int(m.row_ptr[1]), m.gamma) == request_header(rid, 3, **rng)[:3] + (gamma,)
        assert np.array_equal(rp.numpy(), m.row_ptr) and np.array_equal(col.numpy(), m.col)
        assert np.array_equal(g.numpy(), m.g)
        np.testing.assert_allclose(val.numpy(), m.val, rtol=1e-13, atol=0)
        assert m.col.min() >= 0 and m.col.max() < S
        np.testing.assert_allclose(m.val.reshape(-1, k).sum(axis=1), 1.0, rtol=0, atol=1e-14)
        assert np.all(np.diff(m.col.reshape(-1, k), axis=1) >= 0)


def test_request_header_ranges():
    from mdpgen import request_header
    hs = [request_header(r, 5) for r in range(400)]
    S = np.array([h[0] for h in hs])
    assert S.min() >= 1000 and S.max() <= 1_000_000
    assert {h[1] for h in hs} <= set(range(2, 33)) and len({h[1] for h in hs}) > 20
    assert {h[2] for h in hs} <= set(range(4, 65))
    assert {h[3] for h in hs} == {0.9, 0.99, 0.999, 0.9999}
    # log-uniform: about a third of the requests below 1e4
    assert 0.2 < np.mean(S < 10_000) < 0.45


def test_quantize_rows_properties():
    """Largest-remainder rounding (with hypothesis, where installed): every row sums to
    exactly one, holds multiples of 2^-bits only (exact in binary16 for 11 bits and in
    bfloat16 for 8), and moves no entry by a full unit 2^-bits."""
    hyp = pytest.importorskip("hypothesis")
    st = pytest.importorskip("hypothesis.strategies")

    @hyp.settings(max_examples=300, deadline=None, derandomize=True)
    @hyp.given(st.lists(st.floats(1e-6, 1e6), min_size=1, max_size=70), st.sampled_from([8, 11]))
    def check(w, bits):
        w = np.array([w])
        q = quantize_rows(w, bits)[0]
        unit = 2.0 ** bits
        assert q.sum() == 1.0
        assert np.all(q >= 0) and np.all(q * unit == np.round(q * unit))
        assert np.all(np.abs(q - w[0] / w[0].sum()) < 1 / unit)
        import torch
        narrow = torch.float16 if bits == 11 else torch.bfloat16
        assert torch.equal(torch.from_numpy(q).to(narrow).double(), torch.from_numpy(q))

    check()
