"""Device draw of the counter-based serving requests (generators.serving_request_philox)
by a small CUDA kernel, for serving streams whose requests are too large to draw
on the host or with tensor ops in the time of a solve.  Input generation only;
built in-tree for sm_103a like the solver library, loaded with ctypes.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc", "request_gen.cu")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libmdpgen.so")
FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-shared", "-Xcompiler", "-fPIC"]
_lib = None


def build() -> str:
    """Compile libmdpgen.so if the source or flags changed; return its path."""
    h = hashlib.sha256((" ".join(FLAGS)).encode() + open(SRC, "rb").read()).hexdigest()
    stamp = os.path.join(BUILD, "stamp")
    if os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read().strip() == h:
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    tmp = LIB + ".tmp"
    r = subprocess.run([nvcc, *FLAGS, SRC, "-o", tmp], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {SRC}:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(h)
    return LIB


def load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.mdpgen_request.restype = ctypes.c_int
        lib.mdpgen_request.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p]
        _lib = lib
    return _lib


def serving_request_cuda(rid: int, seed: int = 5, s_range=(1_000, 1_000_000), a_range=(2, 32), k_range=(4, 64),
                         gammas=(0.9, 0.99, 0.999, 0.9999), stream=None):
    """(S, A, k, gamma, row_ptr, col, val, g) of request rid, drawn on the current
    CUDA device (torch tensors; the kernel runs on `stream` or torch's current one)."""
    import torch

    from .generators import request_header
    S, A, k, gamma = request_header(rid, seed, s_range, a_range, k_range, gammas)
    R = S * A
    col = torch.empty(R * k, dtype=torch.int32, device="cuda")
    val = torch.empty(R * k, dtype=torch.float64, device="cuda")
    g = torch.empty(R, dtype=torch.float64, device="cuda")
    st = stream if stream is not None else torch.cuda.current_stream()
    rc = load().mdpgen_request(seed & 0xFFFFFFFF, rid, S, A, k, col.data_ptr(), val.data_ptr(), g.data_ptr(),
                               ctypes.c_void_p(st.cuda_stream))
    if rc != 0:
        raise RuntimeError(f"mdpgen_request failed ({rc})")
    row_ptr = torch.arange(R + 1, dtype=torch.int64, device="cuda") * k
    return S, A, k, gamma, row_ptr, col, val, g
