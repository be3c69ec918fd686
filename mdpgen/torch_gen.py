"""The random sparse generator of generators.py, written with torch tensor ops so
it can run on the GPU: same Philox4x32-10 streams, same Floyd column draws, same
Dirichlet weights and quantisation, so the columns and costs are bit for bit
those of `random_sparse`; the weights go through log1p, sqrt, cos and a row
sum, whose last bits may differ between libraries, so probabilities agree to
rounding and quantised ones can differ in rare rows near a rounding boundary.  Used to build the 2e9-entry workload on
the device in seconds instead of half an hour of numpy.  Like the rest of the
package it holds random-number plumbing only, no MDP arithmetic.
"""
from __future__ import annotations

import math

from .generators import REQUEST_ROW_BITS, TAG_COLS, TAG_COST, TAG_VALS, request_header

_M0 = 0xD2511F53
_M1 = 0xCD9E8D57
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK32 = 0xFFFFFFFF


def _mulhilo(a, m: int):
    """High and low 32-bit words of a * m for 32-bit a (int64 tensor) and m, with
    every intermediate below 2**63: a = a_hi 2**16 + a_lo."""
    x = (a & 0xFFFF) * m
    y = (a >> 16) * m
    t = ((y & 0xFFFF) << 16) + x
    return (y >> 16) + (t >> 32), t & _MASK32


def philox4x32(c0, c1, c2, c3, k0: int, k1: int, rounds: int = 10):
    """Philox4x32-R on int64 tensors holding 32-bit words."""
    for r in range(rounds):
        hi0, lo0 = _mulhilo(c0, _M0)
        hi1, lo1 = _mulhilo(c2, _M1)
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        if r + 1 < rounds:
            k0 = (k0 + _W0) & _MASK32
            k1 = (k1 + _W1) & _MASK32
    return c0, c1, c2, c3


def uniform53(hi_word, lo_word):
    import torch
    m = (hi_word >> 5) * (1 << 26) + (lo_word >> 6)
    return m.to(torch.float64) * (2.0 ** -53)


def stream(seed: int, tag: int, row, block, lane: int = 0):
    """Uniform doubles in [0, 1) for (row, block) counters (int64 tensors, row < 2**63)."""
    import torch
    row, block = torch.broadcast_tensors(row, block)
    out = philox4x32(row & _MASK32, row >> 32, block & _MASK32, block >> 32, seed & _MASK32, tag & _MASK32)
    return uniform53(out[0], out[1]) if lane == 0 else uniform53(out[2], out[3])


def _quantize_rows(w, bits: int):
    import torch
    unit = float(1 << bits)
    x = w / w.sum(dim=1, keepdim=True) * unit
    q = torch.floor(x)
    missing = (unit - q.sum(dim=1)).to(torch.int64)
    rem = x - q
    order = torch.argsort(-rem, dim=1, stable=True)
    ranks = torch.empty_like(order)
    ranks.scatter_(1, order, torch.arange(w.shape[1], device=w.device).expand_as(order).contiguous())
    q += (ranks < missing[:, None]).to(torch.float64)
    return q / unit


def random_sparse_device(S: int, A: int, k: int, gamma: float, seed: int, conc: float = 1.0,
                         quant_bits: int | None = None, device="cuda", chunk_rows: int = 1 << 21):
    """Device tensors (row_ptr int64, col int32, val float64, g float64) of
    generators.random_sparse(S, A, k, gamma, seed, conc, quant_bits)."""
    import torch
    if k > S:
        raise ValueError("k > S")
    R = S * A
    col = torch.empty(R * k, dtype=torch.int32, device=device)
    val = torch.empty(R * k, dtype=torch.float64, device=device)
    j = torch.arange(k, dtype=torch.int64, device=device)[None, :]
    for r0 in range(0, R, chunk_rows):
        r1 = min(R, r0 + chunk_rows)
        rows = torch.arange(r0, r1, dtype=torch.int64, device=device)
        # k distinct columns per row (Floyd), sorted
        chosen = torch.empty((r1 - r0, k), dtype=torch.int64, device=device)
        for i in range(k):
            jmax = S - k + i
            u = stream(seed, TAG_COLS, rows, torch.tensor(i, dtype=torch.int64, device=device))
            t = torch.clamp(torch.floor(u * (jmax + 1)).to(torch.int64), max=jmax)
            if i:
                dup = (chosen[:, :i] == t[:, None]).any(dim=1)
                t = torch.where(dup, torch.full_like(t, jmax), t)
            chosen[:, i] = t
        chosen, _ = torch.sort(chosen, dim=1)
        # Dirichlet(conc) weights
        r = rows[:, None]
        if conc == 1.0:
            w = -torch.log1p(-stream(seed, TAG_VALS, r, j))
        elif conc == 0.5:
            u1 = stream(seed, TAG_VALS, r, j, lane=0)
            u2 = stream(seed, TAG_VALS, r, j, lane=1)
            z = torch.sqrt(-2.0 * torch.log1p(-u1)) * torch.cos(2.0 * math.pi * u2)
            w = 0.5 * z * z
            dead = w.sum(dim=1) <= 0.0
            if bool(dead.any()):
                w[dead] = 1.0
        else:
            raise ValueError("supported Dirichlet concentrations: 1.0, 0.5")
        p = w / w.sum(dim=1, keepdim=True) if quant_bits is None else _quantize_rows(w, quant_bits)
        col[r0 * k:r1 * k] = chosen.reshape(-1).to(torch.int32)
        val[r0 * k:r1 * k] = p.reshape(-1)
        del chosen, w, p
    g = stream(seed, TAG_COST, torch.arange(R, dtype=torch.int64, device=device),
               torch.tensor(0, dtype=torch.int64, device=device))
    row_ptr = torch.arange(R + 1, dtype=torch.int64, device=device) * k
    return row_ptr, col, val, g


def serving_request_device(rid: int, seed: int = 5, s_range=(1_000, 1_000_000), a_range=(2, 32), k_range=(4, 64),
                           gammas=(0.9, 0.99, 0.999, 0.9999), device="cuda", chunk_rows: int = 1 << 21):
    """Request rid of generators.serving_request_philox drawn with tensor ops:
    (S, A, k, gamma, row_ptr, col, val, g) with device tensors.  Columns and costs
    equal the numpy draw bit for bit; probabilities agree to rounding."""
    import torch
    S, A, k, gamma = request_header(rid, seed, s_range, a_range, k_range, gammas)
    R = S * A
    col = torch.empty(R * k, dtype=torch.int32, device=device)
    val = torch.empty(R * k, dtype=torch.float64, device=device)
    j = torch.arange(k, dtype=torch.int64, device=device)[None, :]
    base = rid << REQUEST_ROW_BITS
    for r0 in range(0, R, chunk_rows):
        r1 = min(R, r0 + chunk_rows)
        rows = base + torch.arange(r0, r1, dtype=torch.int64, device=device)[:, None]
        u = stream(seed, TAG_COLS, rows, j)
        c = torch.clamp(torch.floor(u * S).to(torch.int64), max=S - 1)
        c, _ = torch.sort(c, dim=1)
        w = -torch.log1p(-stream(seed, TAG_VALS, rows, j + k))
        p = w / w.sum(dim=1, keepdim=True)
        col[r0 * k:r1 * k] = c.reshape(-1).to(torch.int32)
        val[r0 * k:r1 * k] = p.reshape(-1)
        del u, c, w, p
    g = stream(seed, TAG_COST, base + torch.arange(R, dtype=torch.int64, device=device),
               torch.tensor(0, dtype=torch.int64, device=device))
    row_ptr = torch.arange(R + 1, dtype=torch.int64, device=device) * k
    return S, A, k, gamma, row_ptr, col, val, g
