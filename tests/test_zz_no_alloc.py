"""mdp_bellman_csr_noalloc, the entry point for callers that cannot allocate device
memory, against mdp_bellman (the handle-based sweep) on the same inputs.

The file name sorts last so that a run stopping at its first failure has run every
other test first; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from mdpgen import banded_birth_death, random_sparse, random_value_vector
from tests._util import check_policy, q_tolerance, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2507_22538_gb300.build import build
    from paper_2507_22538_gb300 import mdp
    build()
    mdp.load()
    return mdp


@pytest.mark.parametrize("make", [lambda: random_sparse(1037, 5, 8, 0.95, seed=31),
                                  lambda: banded_birth_death(20000, 20, 16, 0.999),
                                  # the largest size the fixed scratch takes: 65536 tiles of 32 states,
                                  # where the last tile's slot sits next to the completion counter
                                  lambda: random_sparse(2_097_152, 2, 2, 0.9, seed=41)],
                         ids=["random_ragged", "banded", "max_states"])
def test_noalloc_matches_bellman_on_two_calls(lib, make):
    import torch
    mdp = lib
    m = make()
    d = to_device(m)
    from oracle import mdp_oracle as O
    P = O.stacked_matrix(m.S, m.A, m.row_ptr, m.col, m.val)
    with mdp.MDP(m.S, m.A, d["row_ptr"], d["col"], d["val"], d["g"]) as M:
        for call, seed in enumerate((3, 4)):  # two calls in a row share the static scratch
            V = torch.from_numpy(random_value_vector(m.S, seed, 1.0 / (1 - m.gamma))).cuda()
            TV_ref, pi_ref, res_ref = M.bellman(m.gamma, V)
            TV = torch.full_like(V, float("nan"))
            pi = torch.full((m.S,), -1, dtype=torch.int32, device="cuda")
            res = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            st = mdp.mdp_bellman_csr_noalloc(m.S, m.A, d["row_ptr"], d["col"], d["val"], d["g"], m.gamma, V, TV,
                                             pi, res)
            assert st == mdp.MDP_OK, mdp.mdp_last_error()
            torch.cuda.synchronize()
            tol = q_tolerance(m, V.cpu().numpy())
            np.testing.assert_allclose(TV.cpu().numpy(), TV_ref.cpu().numpy(), rtol=0, atol=tol)
            assert abs(res.item() - res_ref.item()) <= tol
            # policies: equal wherever the Q gap resolves; elsewhere both attain the minimum
            Q = O.q_values(P, m.g, m.gamma, V.cpu().numpy(), m.S, m.A)
            check_policy(pi.cpu().numpy(), Q, tol)
            check_policy(pi_ref.cpu().numpy(), Q, tol)


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    mdp = lib
    st = mdp.mdp_bellman_csr_noalloc(2_097_153, 4, 1, 1, 1, 1, 0.9, 1, 2, 3, None, stream=0)
    assert st == mdp.MDP_ERR_INVALID_ARG and "2097152" in mdp.mdp_last_error()
    st = mdp.mdp_bellman_csr_noalloc(100, 129, 1, 1, 1, 1, 0.9, 1, 2, 3, None, stream=0)
    assert st == mdp.MDP_ERR_INVALID_ARG and "128" in mdp.mdp_last_error()


def test_noalloc_allocates_nothing(lib):
    """The point of the entry point: once its first call on the device has looked up
    the scratch address, later calls change neither torch's allocator nor the
    device's free memory (cudaMemGetInfo)."""
    import torch
    mdp = lib
    m = random_sparse(5000, 4, 8, 0.9, seed=32)
    d = to_device(m)
    V = torch.from_numpy(random_value_vector(m.S, 5, 10.0)).cuda()
    TV = torch.empty_like(V)
    pi = torch.empty(m.S, dtype=torch.int32, device="cuda")
    res = torch.empty(1, dtype=torch.float64, device="cuda")
    args = (m.S, m.A, d["row_ptr"], d["col"], d["val"], d["g"], m.gamma, V, TV, pi, res)
    assert mdp.mdp_bellman_csr_noalloc(*args) == mdp.MDP_OK, mdp.mdp_last_error()  # first call: set-up
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    for _ in range(3):
        assert mdp.mdp_bellman_csr_noalloc(*args) == mdp.MDP_OK, mdp.mdp_last_error()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0

