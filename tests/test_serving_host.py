"""Host logic of the solve service that needs no GPU: the admission estimate of what
mdp_create holds on the device while it uploads a host MDP in chunks."""
import bisect
import types

import numpy as np
import pytest


def _ring_bytes(row_ptr, cap_entries, buffers):
    """Device bytes of the upload ring as mdp_create sizes it: row-aligned chunks of at
    most cap entries (or one longest row) cut by binary search on the row pointers,
    min(buffers, chunks) buffers of cap entries, 4 B column + 8 B value each."""
    R = len(row_ptr) - 1
    nnz = int(row_ptr[-1] - row_ptr[0])
    kmax = int(np.max(np.diff(row_ptr)))
    cap = min(nnz, max(cap_entries, kmax))
    chunks, r0 = 0, 0
    while r0 < R:
        r1 = bisect.bisect_right(row_ptr, row_ptr[r0] + cap, r0 + 1, R + 1) - 1
        assert r1 > r0 and row_ptr[r1] - row_ptr[r0] <= cap
        chunks, r0 = chunks + 1, r1
    return 12 * cap * min(buffers, chunks)


@pytest.mark.parametrize("seed", range(40))
def test_creation_estimate_bounds_the_upload_ring(monkeypatch, seed):
    from paper_2507_22538_gb300 import serve
    rng = np.random.default_rng(seed)
    S, A = int(rng.integers(1, 60)), int(rng.integers(1, 6))
    lens = rng.integers(1, int(rng.integers(2, 40)), size=S * A)
    row_ptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    cap = int(rng.integers(1, 300))
    monkeypatch.setattr(serve, "UPLOAD_CHUNK_ENTRIES", cap)
    data = types.SimpleNamespace(S=S, A=A, row_ptr=row_ptr)
    est = serve._creation_bytes(S, A, int(row_ptr[-1]), int(lens.max()), True)
    rows = 8 * (S * A + 1) + 4 * S * A
    ring = _ring_bytes(row_ptr, cap, serve.UPLOAD_BUFFERS)
    assert ring <= est - rows
    assert serve.device_bytes(data) > est  # the handle itself comes on top


def test_creation_estimate_large_host_and_device_inputs():
    from paper_2507_22538_gb300 import serve
    S, A, k = 1_000_000, 20, 33
    nnz = S * A * k
    host = serve._creation_bytes(S, A, nnz, k, True)
    dev = serve._creation_bytes(S, A, nnz, k, False)
    rows = 8 * (S * A + 1) + 4 * S * A
    assert host - rows == 12 * serve.UPLOAD_CHUNK_ENTRIES * serve.UPLOAD_BUFFERS  # four chunks, not the CSR
    assert dev - rows == 12 * nnz  # the request's own device CSR
    # a host MDP that fits in one chunk is held whole
    assert serve._creation_bytes(1000, 4, 8000, 8, True) - (8 * 4001 + 4 * 4000) == 12 * 8000
