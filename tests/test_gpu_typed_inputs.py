"""mdp_create from P values in binary32, binary16 or bfloat16 (mdp_dtype): the
library widens each value exactly to binary64, so an MDP whose probabilities are
exact in the narrow type gives the same handle as the binary64 input and the same
results bit for bit (the binary64 path is checked against the oracle elsewhere);
values that do not make stochastic rows after widening are rejected."""
import numpy as np
import pytest

from mdpgen import banded_birth_death, random_sparse, random_value_vector

pytestmark = pytest.mark.gpu


def _typed(val, dtype):
    import torch
    t = torch.from_numpy(val)
    return {"f32": t.to(torch.float32), "f16": t.to(torch.float16), "bf16": t.to(torch.bfloat16)}[dtype]


CASES = [
    ("random_f16", lambda: random_sparse(2000, 6, 9, 0.95, seed=3, quant_bits=11), "f16"),
    ("banded_f16", lambda: banded_birth_death(4000, 20, 16, 0.999, quant_bits=11), "f16"),
    ("random_bf16", lambda: random_sparse(1500, 5, 7, 0.9, seed=4, quant_bits=8), "bf16"),
    ("random_f32", lambda: random_sparse(1800, 4, 12, 0.95, seed=5, quant_bits=11), "f32"),
]


@pytest.mark.parametrize("on_device", [False, True], ids=["host", "device"])
@pytest.mark.parametrize("name,make,dtype", CASES, ids=[c[0] for c in CASES])
def test_narrow_values_give_the_binary64_results(name, make, dtype, on_device):
    import torch
    from paper_2507_22538_gb300 import mdp
    m = make()
    narrow = _typed(m.val, dtype)
    assert torch.equal(narrow.to(torch.float64), torch.from_numpy(m.val))  # exact in the narrow type
    if on_device:
        args = [torch.from_numpy(m.row_ptr).cuda(), torch.from_numpy(m.col).cuda(), narrow.cuda(),
                torch.from_numpy(m.g).cuda()]
    else:
        args = [m.row_ptr, m.col, narrow.pin_memory(), m.g]
    V = torch.from_numpy(random_value_vector(m.S, 2, 1.0 / (1 - m.gamma))).cuda()
    with mdp.MDP.from_data(m) as M64, mdp.MDP(m.S, m.A, *args) as Mn:
        for a, b in zip(M64.bellman(m.gamma, V), Mn.bellman(m.gamma, V)):
            assert torch.equal(a, b)
        for prec in (mdp.MDP_PREC_F64, mdp.MDP_PREC_MIXED):
            r64 = M64.solve(m.gamma, tol=1e-9, alpha=1e-3, precision=prec)
            rn = Mn.solve(m.gamma, tol=1e-9, alpha=1e-3, precision=prec)
            torch.cuda.synchronize()
            assert torch.equal(r64[0], rn[0]) and torch.equal(r64[1], rn[1])
            assert (r64[2].outer_iters, r64[2].inner_iters_total) == (rn[2].outer_iters, rn[2].inner_iters_total)
            assert r64[2].policy_value_bytes == rn[2].policy_value_bytes


@pytest.mark.parametrize("bad", ["negative", "nan", "inf", "rounded_f32", "rounded_f16", "bad_type"])
def test_narrow_values_are_validated(bad):
    import torch
    from paper_2507_22538_gb300 import mdp
    m = random_sparse(300, 3, 5, 0.9, seed=6, quant_bits=11)
    val = torch.from_numpy(m.val).to(torch.float16)
    vt = None
    expect = mdp.MDP_ERR_NOT_STOCHASTIC
    pos = int(np.flatnonzero(m.val > 0)[3])  # a nonzero entry (quantised rows may hold explicit zeros)
    if bad == "negative":
        val[pos] = -val[pos]
    elif bad == "nan":
        val[9] = float("nan")
    elif bad == "inf":
        val[9] = float("inf")
    elif bad == "rounded_f32":
        # Dirichlet(1) probabilities rounded to binary32: rows miss 1 by more than 1e-12
        val = torch.from_numpy(random_sparse(300, 3, 5, 0.9, seed=6).val).to(torch.float32)
    elif bad == "rounded_f16":
        val = torch.from_numpy(random_sparse(300, 3, 5, 0.9, seed=6).val).to(torch.float16)
    elif bad == "bad_type":
        vt, expect = 7, mdp.MDP_ERR_INVALID_ARG
    st, h = mdp.mdp_create(m.S, m.A, m.row_ptr, m.col, val, m.g, False, stream=0, val_type=vt)
    assert st == expect, (st, mdp.mdp_last_error())
    assert not h.value
