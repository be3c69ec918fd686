"""Thin ctypes binding of libmdp (include/mdp.h): argument marshalling only.

The functions keep the C names and return the C status codes; every
computation runs in the library's CUDA kernels.  Arrays may be torch tensors
(device or host) or numpy arrays (host); streams are torch.cuda.Stream
objects, raw cudaStream_t integers, or None for the current torch stream.

The library must be built first (``paper_2507_22538_gb300.build.build()``);
loading fails loudly when it is missing.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmdp.so")

MDP_OK = 0
MDP_ERR_INVALID_ARG = 1
MDP_ERR_NOT_STOCHASTIC = 2
MDP_ERR_OOM = 3
MDP_ERR_CUDA = 4
MDP_NOT_CONVERGED = 5
MDP_ERR_NUMERIC = 6
STATUS_NAMES = {0: "MDP_OK", 1: "MDP_ERR_INVALID_ARG", 2: "MDP_ERR_NOT_STOCHASTIC", 3: "MDP_ERR_OOM",
                4: "MDP_ERR_CUDA", 5: "MDP_NOT_CONVERGED", 6: "MDP_ERR_NUMERIC"}

MDP_F64, MDP_F32, MDP_F16, MDP_BF16 = 0, 1, 2, 3  # mdp_dtype: storage type of the P values
MDP_GMRES = 0
MDP_RICHARDSON = 1
MDP_TFQMR = 2
MDP_RICHARDSON_JACOBI = 3
MDP_REFINE_NEVER = 0
MDP_REFINE_IFNEEDED = 1
MDP_REFINE_ALWAYS = 2
MDP_PREC_F64 = 0
MDP_PREC_MIXED = 1


class mdp_solve_opts(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("atol_pi", ctypes.c_double), ("alpha", ctypes.c_double),
                ("richardson_scale", ctypes.c_double), ("max_iter_pi", ctypes.c_int32),
                ("max_iter_ksp", ctypes.c_int32), ("gmres_restart", ctypes.c_int32), ("inner", ctypes.c_int32),
                ("record_timing", ctypes.c_int32), ("gmres_refine", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("graph", ctypes.c_int32), ("lowp_sweep", ctypes.c_int32)]


class mdp_solve_stats(ctypes.Structure):
    _fields_ = [("outer_iters", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("inner_iters_total", ctypes.c_int64), ("final_residual", ctypes.c_double),
                ("seconds", ctypes.c_double), ("kernel_launches", ctypes.c_int64),
                ("bellman_sweeps", ctypes.c_int32), ("bellman_ms", ctypes.c_double),
                ("inner_ms", ctypes.c_double), ("policy_matvecs", ctypes.c_int64),
                ("vector_reads", ctypes.c_int64), ("vector_writes", ctypes.c_int64), ("inner_bytes", ctypes.c_double),
                ("policy_value_bytes", ctypes.c_int32), ("matvec_ms", ctypes.c_double),
                ("matvecs_timed", ctypes.c_int64), ("gs_ms", ctypes.c_double), ("gs_flops", ctypes.c_double),
                ("gs_timed", ctypes.c_int64), ("bellman_value_bytes", ctypes.c_int32),
                ("bellman_rows_fp64", ctypes.c_int64), ("matvec_bytes", ctypes.c_double),
                ("matvec_flops", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None

_P = ctypes.c_void_p
_SIGNATURES = {
    "mdp_default_opts": (None, [ctypes.POINTER(mdp_solve_opts)]),
    "mdp_create": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, _P, _P, _P, ctypes.c_int, _P, ctypes.c_int32, _P,
                                  ctypes.POINTER(_P)]),
    "mdp_destroy": (ctypes.c_int, [_P]),
    "mdp_get_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32),
                                    ctypes.POINTER(ctypes.c_int64)]),
    "mdp_bellman": (ctypes.c_int, [_P, ctypes.c_double, _P, _P, _P, _P, _P]),
    "mdp_bellman_lowp": (ctypes.c_int, [_P, ctypes.c_double, _P, _P, _P, _P, _P]),
    "mdp_policy_apply": (ctypes.c_int, [_P, ctypes.c_double, _P, _P, _P, _P]),
    "mdp_policy_eval": (ctypes.c_int, [_P, ctypes.c_double, _P, _P, _P, ctypes.c_int, ctypes.c_int32,
                                       ctypes.c_double, ctypes.c_double, ctypes.c_int32,
                                       ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_double), _P]),
    "mdp_solve": (ctypes.c_int, [_P, ctypes.POINTER(mdp_solve_opts), _P, _P, ctypes.POINTER(mdp_solve_stats), _P]),
    "mdp_solve_batch": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(_P), ctypes.POINTER(mdp_solve_opts),
                                       ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(mdp_solve_stats),
                                       ctypes.POINTER(ctypes.c_int), _P]),
    "mdp_solve_small_batch": (ctypes.c_int, [ctypes.c_int32, ctypes.POINTER(_P), ctypes.POINTER(mdp_solve_opts),
                                             ctypes.POINTER(_P), ctypes.POINTER(_P), ctypes.POINTER(mdp_solve_stats),
                                             ctypes.POINTER(ctypes.c_int), _P]),
    "mdp_tune": (ctypes.c_int, [_P, ctypes.c_double, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_float),
                                _P]),
    "mdp_get_sweep_shape": (ctypes.c_int, [_P] + [ctypes.POINTER(ctypes.c_int32)] * 5),
    "mdp_set_sweep_shape": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]),
    "mdp_last_error": (ctypes.c_char_p, []),
    "mdp_bellman_csr_noalloc": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, _P, _P, _P, _P, ctypes.c_double,
                                               _P, _P, _P, _P, _P]),
}


def load(path: str = LIB_PATH):
    """Load libmdp.so (once) and declare the C signatures."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"libmdp.so is not built ({path}); run paper_2507_22538_gb300.build.build()")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


class MDPError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {mdp_last_error()}")


def check(status: int, where: str, allow=(MDP_OK,)):
    if status not in allow:
        raise MDPError(status, where)
    return status


# ---- the C entry points, same names ------------------------------------------------

def mdp_default_opts() -> mdp_solve_opts:
    o = mdp_solve_opts()
    load().mdp_default_opts(ctypes.byref(o))
    return o


def mdp_last_error() -> str:
    return load().mdp_last_error().decode()


def value_dtype(val) -> int:
    """The mdp_dtype of a numpy array or torch tensor of P values."""
    name = str(getattr(val, "dtype", "float64")).replace("torch.", "")
    codes = {"float64": MDP_F64, "float32": MDP_F32, "float16": MDP_F16, "bfloat16": MDP_BF16}
    if name not in codes:
        raise TypeError(f"P values of dtype {name}: expected float64, float32, float16 or bfloat16")
    return codes[name]


def mdp_create(S, A, row_ptr, col, val, g, inputs_on_device: bool, stream=None, val_type=None):
    """Returns (status, handle).  val_type defaults to the dtype of val."""
    h = _P()
    vt = value_dtype(val) if val_type is None else int(val_type)
    st = load().mdp_create(int(S), int(A), _ptr(row_ptr), _ptr(col), _ptr(val), vt, _ptr(g),
                           1 if inputs_on_device else 0, _stream(stream), ctypes.byref(h))
    return st, h


def mdp_destroy(h) -> int:
    return load().mdp_destroy(h)


def mdp_get_info(h):
    S, A, nnz = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64()
    st = load().mdp_get_info(h, ctypes.byref(S), ctypes.byref(A), ctypes.byref(nnz))
    return st, S.value, A.value, nnz.value


def mdp_bellman(h, gamma, V, TV, pi, residual_inf=None, stream=None) -> int:
    return load().mdp_bellman(h, float(gamma), _ptr(V), _ptr(TV), _ptr(pi), _ptr(residual_inf), _stream(stream))


def mdp_bellman_lowp(h, gamma, V, TV, pi, residual_inf=None, stream=None) -> int:
    return load().mdp_bellman_lowp(h, float(gamma), _ptr(V), _ptr(TV), _ptr(pi), _ptr(residual_inf),
                                   _stream(stream))


def mdp_policy_apply(h, gamma, pi, x, y, stream=None) -> int:
    return load().mdp_policy_apply(h, float(gamma), _ptr(pi), _ptr(x), _ptr(y), _stream(stream))


def mdp_policy_eval(h, gamma, pi, v0, v, inner=MDP_GMRES, restart=30, omega=1.0, abs_tol_2norm=1e-10,
                    max_it=1000, stream=None):
    """Returns (status, iterations, residual 2-norm)."""
    it, res = ctypes.c_int32(), ctypes.c_double()
    st = load().mdp_policy_eval(h, float(gamma), _ptr(pi), _ptr(v0), _ptr(v), int(inner), int(restart),
                                float(omega), float(abs_tol_2norm), int(max_it), ctypes.byref(it),
                                ctypes.byref(res), _stream(stream))
    return st, it.value, res.value


def mdp_solve(h, opts: mdp_solve_opts, V, pi, stream=None):
    """Returns (status, mdp_solve_stats)."""
    stats = mdp_solve_stats()
    st = load().mdp_solve(h, ctypes.byref(opts), _ptr(V), _ptr(pi), ctypes.byref(stats), _stream(stream))
    return st, stats


def mdp_tune(h, gamma, stream=None):
    """Returns (status, chosen tile size, ms per sweep)."""
    ts = ctypes.c_int32(0)
    ms = ctypes.c_float(0.0)
    st = load().mdp_tune(h, float(gamma), ctypes.byref(ts), ctypes.byref(ms), _stream(stream))
    return st, ts.value, ms.value


def mdp_set_sweep_shape(h, tile_states, rows_per_warp=32, value_load_bytes=16, blocks_per_sm=0):
    return load().mdp_set_sweep_shape(h, int(tile_states), int(rows_per_warp), int(value_load_bytes),
                                      int(blocks_per_sm))


def mdp_get_sweep_shape(h):
    """(status, {tile_states, blocks, blocks_per_sm, rows_per_warp, value_load_bytes}) of the
    handle's Bellman sweep."""
    v = [ctypes.c_int32() for _ in range(5)]
    st = load().mdp_get_sweep_shape(h, *[ctypes.byref(x) for x in v])
    return st, dict(zip(("tile_states", "blocks", "blocks_per_sm", "rows_per_warp", "value_load_bytes"),
                        (x.value for x in v)))


def mdp_solve_batch(handles, opts, V, pi, stream=None):
    """Solve len(handles) MDPs in lockstep.  opts: a list of mdp_solve_opts; V, pi:
    lists of device tensors.  Returns (status of the call, [per-problem status],
    [per-problem mdp_solve_stats])."""
    n = len(handles)
    if not (len(opts) == len(V) == len(pi) == n):
        raise ValueError("handles, opts, V and pi must have the same length")
    hs = (_P * n)(*handles)
    os_ = (mdp_solve_opts * n)(*opts)
    vs = (_P * n)(*[_ptr(v) for v in V])
    ps = (_P * n)(*[_ptr(p) for p in pi])
    stats = (mdp_solve_stats * n)()
    status = (ctypes.c_int * n)()
    st = load().mdp_solve_batch(n, hs, os_, vs, ps, stats, status, _stream(stream))
    return st, list(status), list(stats)


def mdp_solve_small_batch(handles, opts, V, pi, stream=None):
    """Solve len(handles) small MDPs, one thread-block cluster each, in one launch per
    cluster size.  Same arguments and returns as mdp_solve_batch."""
    n = len(handles)
    if not (len(opts) == len(V) == len(pi) == n):
        raise ValueError("handles, opts, V and pi must have the same length")
    hs = (_P * n)(*handles)
    os_ = (mdp_solve_opts * n)(*opts)
    vs = (_P * n)(*[_ptr(v) for v in V])
    ps = (_P * n)(*[_ptr(p) for p in pi])
    stats = (mdp_solve_stats * n)()
    status = (ctypes.c_int * n)()
    st = load().mdp_solve_small_batch(n, hs, os_, vs, ps, stats, status, _stream(stream))
    return st, list(status), list(stats)


def mdp_bellman_csr_noalloc(S, A, row_ptr, col, val, g, gamma, V, TV, pi, residual_inf=None, stream=None) -> int:
    """Bellman application from device CSR arrays without a handle or any device allocation."""
    return load().mdp_bellman_csr_noalloc(int(S), int(A), _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(g),
                                          float(gamma), _ptr(V), _ptr(TV), _ptr(pi), _ptr(residual_inf),
                                          _stream(stream))


# ---- a small convenience wrapper over torch device buffers --------------------------

class MDP:
    """Owns an mdp_handle; inputs are host numpy arrays or device torch tensors."""

    def __init__(self, S, A, row_ptr, col, val, g, stream=None):
        import torch
        on_dev = isinstance(row_ptr, torch.Tensor) and row_ptr.is_cuda
        st, self.h = mdp_create(S, A, row_ptr, col, val, g, on_dev, stream)
        check(st, "mdp_create")
        self.S, self.A = int(S), int(A)

    @classmethod
    def from_data(cls, m, stream=None):
        return cls(m.S, m.A, m.row_ptr, m.col, m.val, m.g, stream)

    def close(self):
        if self.h:
            mdp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def bellman(self, gamma, V, stream=None):
        import torch
        TV = torch.empty_like(V)
        pi = torch.empty(self.S, dtype=torch.int32, device=V.device)
        res = torch.empty(1, dtype=torch.float64, device=V.device)
        check(mdp_bellman(self.h, gamma, V, TV, pi, res, stream), "mdp_bellman")
        return TV, pi, res

    def bellman_lowp(self, gamma, V, stream=None):
        import torch
        TV = torch.empty_like(V)
        pi = torch.empty(self.S, dtype=torch.int32, device=V.device)
        res = torch.empty(1, dtype=torch.float64, device=V.device)
        check(mdp_bellman_lowp(self.h, gamma, V, TV, pi, res, stream), "mdp_bellman_lowp")
        return TV, pi, res

    def policy_apply(self, gamma, pi, x, stream=None):
        import torch
        y = torch.empty_like(x)
        check(mdp_policy_apply(self.h, gamma, pi, x, y, stream), "mdp_policy_apply")
        return y

    def policy_eval(self, gamma, pi, v0, inner=MDP_GMRES, restart=30, omega=1.0, tol=1e-10, max_it=1000,
                    stream=None):
        import torch
        v = torch.empty_like(v0)
        st, it, res = mdp_policy_eval(self.h, gamma, pi, v0, v, inner, restart, omega, tol, max_it, stream)
        check(st, "mdp_policy_eval", allow=(MDP_OK, MDP_NOT_CONVERGED))
        return v, it, res, st

    def solve(self, gamma, V0=None, tol=1e-8, alpha=1e-4, inner=MDP_GMRES, restart=30, omega=1.0,
              max_outer=1000, max_inner=1000, record_timing=False, refine=MDP_REFINE_NEVER, precision=MDP_PREC_F64,
              stream=None, device="cuda", graph=False, lowp_sweep=False):
        import torch
        o = mdp_default_opts()
        o.gamma, o.atol_pi, o.alpha, o.richardson_scale = gamma, tol, alpha, omega
        o.max_iter_pi, o.max_iter_ksp, o.gmres_restart, o.inner = max_outer, max_inner, restart, inner
        o.record_timing = 1 if record_timing else 0
        o.gmres_refine = refine
        o.precision = precision
        o.graph = 1 if graph else 0
        o.lowp_sweep = 1 if lowp_sweep else 0
        V = torch.zeros(self.S, dtype=torch.float64, device=device) if V0 is None else V0.clone()
        pi = torch.empty(self.S, dtype=torch.int32, device=V.device)
        st, stats = mdp_solve(self.h, o, V, pi, stream)
        check(st, "mdp_solve", allow=(MDP_OK, MDP_NOT_CONVERGED))
        return V, pi, stats, st
