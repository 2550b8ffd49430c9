"""CPU oracle for the dynamic-graph random walk (FlowWalker, arXiv 2404.08364).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the CPU
baseline leg of the benchmark may import this package; the library itself
never does.  It shares no code with the CUDA path.

``oracle.c`` is a plain single-threaded C walker (Alg. 1 with the weight rules
of Section 2.1, Eq. 1 and Eq. 2) with its own Philox-4x32-10; this module only
builds it with gcc and marshals numpy arrays through ctypes.

Parity pins: every function here is pinned by ``tests/test_oracle_*.py``
against brute force in exact rational arithmetic, closed forms and published
known-answer vectors.  The fast-mode worked examples of Section 4 (Fig. 4) are
parity unpinned: the figure's weights are not in the paper's text.
"""

from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")

WEIGHTED, NODE2VEC, METAPATH, PPR = 0, 1, 2, 3
ALGOS = {"weighted": WEIGHTED, "node2vec": NODE2VEC, "metapath": METAPATH, "ppr": PPR}


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (gcc, portable flags)."""
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-Wall", "-Wextra",
                           "-o", tmp, src])
    os.replace(tmp, _SO)
    return _SO


class _Params(ctypes.Structure):
    _fields_ = [
        ("n2v_ret_i", ctypes.c_uint32), ("n2v_in_i", ctypes.c_uint32), ("n2v_out_i", ctypes.c_uint32),
        ("n2v_ret", ctypes.c_float), ("n2v_in", ctypes.c_float), ("n2v_out", ctypes.c_float),
        ("schema_len", ctypes.c_int32), ("schema", ctypes.c_int8 * 16),
        ("ppr_stop", ctypes.c_double),
    ]


@dataclasses.dataclass
class Params:
    """Walk parameters.  node2vec p (return) and q (in-out) are the paper's
    a and b of Eq. 2; the exact-mode factors are S/p, S, S/q for scale S."""
    p: float = 1.0
    q: float = 1.0
    scale: int = 2
    schema: Sequence[int] = (0, 1, 2, 3, 4)
    ppr_stop: float = 0.2

    def to_c(self) -> _Params:
        c = _Params()
        ret, inn, out = self.scale / self.p, float(self.scale), self.scale / self.q
        for v in (ret, inn, out):
            if v != int(v) or v <= 0:
                raise ValueError("exact-mode node2vec factors must be positive integers")
        c.n2v_ret_i, c.n2v_in_i, c.n2v_out_i = int(ret), int(inn), int(out)
        c.n2v_ret, c.n2v_in, c.n2v_out = 1.0 / self.p, 1.0, 1.0 / self.q
        if not 0 < len(self.schema) <= 16:
            raise ValueError("schema length must be in [1, 16]")
        c.schema_len = len(self.schema)
        for i, s in enumerate(self.schema):
            c.schema[i] = int(s)
        c.ppr_stop = float(self.ppr_stop)
        return c


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(_SO):
            build()
        L = ctypes.CDLL(_SO)
        P = ctypes.c_void_p
        L.orc_philox4x32_10.argtypes = [P, P, P]
        L.orc_philox4x32_10.restype = None
        L.orc_pick.argtypes = [P, ctypes.c_int64, ctypes.c_uint64]
        L.orc_pick.restype = ctypes.c_int64
        L.orc_scale_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        L.orc_scale_draw.restype = ctypes.c_uint64
        L.orc_ppr_threshold.argtypes = [ctypes.c_double]
        L.orc_ppr_threshold.restype = ctypes.c_uint32
        L.orc_walk_exact.argtypes = [ctypes.c_int64, P, P, P, P, ctypes.c_int, ctypes.POINTER(_Params),
                                     P, ctypes.c_int64, ctypes.c_int64, P, ctypes.c_int32,
                                     ctypes.c_uint64, P, P, P, P]
        L.orc_walk_exact.restype = ctypes.c_int
        L.orc_transition.argtypes = [P, P, P, P, P, ctypes.c_int, ctypes.POINTER(_Params), ctypes.c_int,
                                     ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P, P]
        L.orc_transition.restype = ctypes.c_int64
        _lib = L
    return _lib


def _np(x, dtype):
    if x is None:
        return None
    if hasattr(x, "detach"):
        x = x.detach().cpu().numpy()
    a = np.ascontiguousarray(x)
    if a.dtype != np.dtype(dtype):
        if np.dtype(dtype) == np.uint32 and a.dtype == np.int32:
            a = a.view(np.uint32)
        else:
            a = a.astype(dtype)
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


class CSR:
    """Host copy of a graph as numpy arrays (row_ptr, col, w_u32, w_f32, etype)."""

    def __init__(self, g):
        self.n = int(g.n)
        self.row_ptr = _np(g.row_ptr, np.int64)
        self.col = _np(g.col, np.int32)
        self.w_u32 = _np(g.w_u32, np.uint32)
        self.w_f32 = _np(g.w_f32, np.float32)
        self.etype = _np(getattr(g, "etype", None), np.int8)


def philox4x32_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return [int(v) for v in o]


def pick(wp, r: int) -> int:
    a = np.ascontiguousarray(wp, dtype=np.uint64)
    return int(lib().orc_pick(_ptr(a), len(a), r))


def scale_draw(x: int, W: int) -> int:
    return int(lib().orc_scale_draw(x, W))


def ppr_threshold(p_stop: float) -> int:
    return int(lib().orc_ppr_threshold(p_stop))


def walk_exact(csr: CSR, algo, params: Params, starts, max_len: int, seed: int,
               lengths=None, prev=None, step0=None, q0: int = 0):
    """Exact-mode walks; returns (paths int32 [n_q, max_len+1], path_len int32 [n_q])."""
    algo = ALGOS.get(algo, algo)
    st = _np(starts, np.int32)
    n_q = len(st)
    paths = np.empty((n_q, max_len + 1), dtype=np.int32)
    plen = np.empty(n_q, dtype=np.int32)
    ln, pv, s0 = _np(lengths, np.int32), _np(prev, np.int32), _np(step0, np.int32)
    cp = params.to_c()
    rc = lib().orc_walk_exact(csr.n, _ptr(csr.row_ptr), _ptr(csr.col), _ptr(csr.w_u32), _ptr(csr.etype),
                              algo, ctypes.byref(cp), _ptr(st), n_q, q0, _ptr(ln), max_len, seed,
                              _ptr(pv), _ptr(s0), _ptr(paths), _ptr(plen))
    if rc != 0:
        raise ValueError(f"orc_walk_exact failed: {rc}")
    return paths, plen


def transition(csr: CSR, algo, params: Params, cur: int, prev: int = -1, t: int = 0,
               mode: str = "exact"):
    """Transition weights from state (cur, prev, t): uint64 array (exact) or
    float64 array (fast); probabilities are weights / weights.sum()."""
    algo = ALGOS.get(algo, algo)
    d = int(csr.row_ptr[cur + 1] - csr.row_ptr[cur])
    we = np.zeros(max(d, 1), dtype=np.uint64)
    wf = np.zeros(max(d, 1), dtype=np.float64)
    cp = params.to_c()
    lib().orc_transition(_ptr(csr.row_ptr), _ptr(csr.col), _ptr(csr.w_u32), _ptr(csr.w_f32),
                         _ptr(csr.etype), algo, ctypes.byref(cp), 0 if mode == "exact" else 1,
                         cur, prev, t, _ptr(we), _ptr(wf))
    return we[:d] if mode == "exact" else wf[:d]
