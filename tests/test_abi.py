"""The C-ABI library loads here (no GPU) and exports every function include/mdp.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2507_22538_gb300.build import build
    from paper_2507_22538_gb300 import mdp
    build()
    return mdp.load()


def _declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            for m in re.finditer(r"^\s*(?:const\s+)?\w+\s*\*?\s+(mdp_\w+)\s*\(", text, flags=re.M):
                names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = _declared_functions()
    for n in ("mdp_create", "mdp_destroy", "mdp_bellman", "mdp_policy_eval", "mdp_solve", "mdp_last_error",
              "mdp_policy_apply", "mdp_default_opts", "mdp_get_info"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for n in _declared_functions():
        assert hasattr(lib, n), n
        assert isinstance(getattr(lib, n), ctypes._CFuncPtr)


def test_host_only_calls(lib):
    from paper_2507_22538_gb300 import mdp
    o = mdp.mdp_default_opts()
    assert (o.atol_pi, o.alpha, o.richardson_scale) == (1e-8, 1e-4, 1.0)  # Table 1 defaults
    assert (o.max_iter_pi, o.max_iter_ksp, o.gmres_restart, o.inner) == (1000, 1000, 30, mdp.MDP_GMRES)
    assert o.gmres_refine == mdp.MDP_REFINE_NEVER  # PETSc's KSPGMRES default
    assert o.precision == mdp.MDP_PREC_F64
    # argument checks that return before touching the device
    st, h = mdp.mdp_create(0, 4, 1, 1, 1, 1, False, stream=0)
    assert st == mdp.MDP_ERR_INVALID_ARG and not h.value
    assert "S >= 1" in mdp.mdp_last_error()
    assert mdp.mdp_destroy(None) == mdp.MDP_OK
    assert mdp.mdp_bellman(None, 0.9, 1, 2, 3, None, stream=0) == mdp.MDP_ERR_INVALID_ARG


def test_struct_layouts_match_header():
    from paper_2507_22538_gb300 import mdp
    assert ctypes.sizeof(mdp.mdp_solve_opts) == 4 * 8 + 7 * 4 + 4  # padded to 8
    assert ctypes.sizeof(mdp.mdp_solve_stats) == 4 + 4 + 8 + 8 + 8 + 8 + 4 + 4 + 8 + 8 + 3 * 8 + 8 + 4 + 4
