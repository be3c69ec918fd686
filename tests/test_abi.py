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


def test_struct_layouts_match_header(tmp_path):
    """Every field offset and the size of the option and statistics structs, as
    the C compiler lays them out from include/mdp.h, equal the ctypes mirror's."""
    import shutil
    import subprocess

    from paper_2507_22538_gb300 import mdp
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    inc = os.path.join(ROOT, "include")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "mdp.h"', "int main(void) {"]
    for st in (mdp.mdp_solve_opts, mdp.mdp_solve_stats):
        lines.append(f'  printf("{st.__name__} sizeof %zu\\n", sizeof({st.__name__}));')
        for f, _ in st._fields_:
            lines.append(f'  printf("{st.__name__} {f} %zu\\n", offsetof({st.__name__}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", inc, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    c = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for st in (mdp.mdp_solve_opts, mdp.mdp_solve_stats):
        assert c[(st.__name__, "sizeof")] == ctypes.sizeof(st), st.__name__
        for f, _ in st._fields_:
            assert c[(st.__name__, f)] == getattr(st, f).offset, (st.__name__, f)


def test_noalloc_rejects_overlapping_buffers(lib):
    """mdp_bellman_csr_noalloc refuses outputs that share bytes with each other or with
    V, g or row_ptr on the host, before it touches the device (the addresses below are
    never dereferenced; without a GPU a missed overlap would end in a CUDA error, not
    in a launch)."""
    from paper_2507_22538_gb300 import mdp
    S, A = 100, 3
    base = 1 << 20
    V, g, rp = base, base + 10_000, base + 20_000
    TV, pi, res = base + 40_000, base + 50_000, base + 60_000
    for bad in (dict(TV=V + 8), dict(TV=g + S * A * 8 - 8), dict(pi=rp), dict(res=TV + 8 * (S - 1)),
                dict(pi=TV + 4), dict(res=pi + 4 * S - 4)):
        a = dict(V=V, TV=TV, pi=pi, res=res)
        a.update(bad)
        st = mdp.mdp_bellman_csr_noalloc(S, A, rp, 7, 7, g, 0.9, a["V"], a["TV"], a["pi"], a["res"], stream=0)
        assert st == mdp.MDP_ERR_INVALID_ARG and "overlap" in mdp.mdp_last_error(), bad


@pytest.mark.parametrize("args,msg", [
    (dict(S=0, A=4), "S >= 1"),
    (dict(S=10, A=0), "A <= 8192"),
    (dict(S=10, A=8193), "A <= 8192"),
    (dict(S=1 << 31, A=1), "S must fit int32"),
    (dict(S=1 << 30, A=128), "S*A must be below 2^36"),
    (dict(S=10, A=4, row_ptr=0), "null input array"),
    (dict(S=10, A=4, g=0), "null input array"),
    (dict(S=10, A=4, val_type=7), "val_type"),
], ids=["S0", "A0", "A_big", "S_big", "SA_big", "null_row_ptr", "null_g", "val_type"])
def test_create_argument_checks(lib, args, msg):
    """mdp_create refuses bad sizes, null arrays and unknown value types on the host,
    before it touches the device (the addresses below are never dereferenced)."""
    from paper_2507_22538_gb300 import mdp
    a = dict(S=10, A=4, row_ptr=1 << 20, col=1 << 21, val=1 << 22, g=1 << 23, val_type=mdp.MDP_F64)
    a.update(args)
    st, h = mdp.mdp_create(a["S"], a["A"], a["row_ptr"], a["col"], a["val"], a["g"], False, stream=0,
                           val_type=a["val_type"])
    assert st == mdp.MDP_ERR_INVALID_ARG and not h.value
    assert msg in mdp.mdp_last_error(), mdp.mdp_last_error()


def test_null_handles_are_refused(lib):
    """Every handle-taking entry point answers a null handle with MDP_ERR_INVALID_ARG
    and a message, without touching the device."""
    from paper_2507_22538_gb300 import mdp
    o = mdp.mdp_default_opts()
    o.gamma = 0.9
    calls = {
        "mdp_get_info": lambda: mdp.mdp_get_info(None)[0],
        "mdp_bellman_lowp": lambda: mdp.mdp_bellman_lowp(None, 0.9, 1, 2, 3, stream=0),
        "mdp_policy_apply": lambda: mdp.mdp_policy_apply(None, 0.9, 1, 2, 3, stream=0),
        "mdp_policy_eval": lambda: mdp.mdp_policy_eval(None, 0.9, 1, 2, 3, stream=0)[0],
        "mdp_solve": lambda: mdp.mdp_solve(None, o, 1, 2, stream=0)[0],
        "mdp_tune": lambda: mdp.mdp_tune(None, 0.9, stream=0)[0],
        "mdp_set_sweep_shape": lambda: mdp.mdp_set_sweep_shape(None, 64),
        "mdp_get_sweep_shape": lambda: mdp.mdp_get_sweep_shape(None)[0],
        "mdp_solve_batch": lambda: mdp.mdp_solve_batch([None], [o], [1], [2], stream=0)[0],
        "mdp_solve_small_batch": lambda: mdp.mdp_solve_small_batch([None], [o], [1], [2], stream=0)[0],
        "mdp_solve_batch_empty": lambda: mdp.mdp_solve_batch([], [], [], [], stream=0)[0],
        "mdp_solve_small_batch_empty": lambda: mdp.mdp_solve_small_batch([], [], [], [], stream=0)[0],
    }
    for name, call in calls.items():
        assert call() == mdp.MDP_ERR_INVALID_ARG, name
        assert mdp.mdp_last_error(), name


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    """Without libmdp.so the binding raises: there is no other path to fall back on."""
    from paper_2507_22538_gb300 import mdp
    monkeypatch.setattr(mdp, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        mdp.load(str(tmp_path / "libmdp.so"))
