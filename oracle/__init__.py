"""LLP oracle — test infrastructure only.

Plain sequential CPU implementations (``oracle.c``, built with gcc, and the
fp64 numpy MLP in ``mlp.py``) of what each LLP problem converges to.  Only the
tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg import
this package; the product path (``paper_2603_13147_b300``) never does, and this
package imports nothing from it.

Each wrapper takes host numpy arrays laid out like the inputs of the C ABI and
returns numpy arrays.  See ``oracle.c`` for the definitions and citations.
Parity status: every function here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` (paper examples, brute force on tiny inputs,
closed forms, invariants).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

INF = 0xFFFFFFFF
OK, ERR_ARG, ERR_INFEASIBLE, ERR_OVERFLOW, ERR_CYCLE = 0, 1, 5, 6, 8


def build(force: bool = False) -> str:
    """Compile oracle.c (plain C, -O2, no OpenMP: the oracle is sequential)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            lib.oracle_sum_u64.restype = ctypes.c_uint64
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"oracle {what}: status {code}")
        self.code = code


def sssp(offsets, indices, weights, source: int, check: bool = True) -> np.ndarray:
    """Dijkstra distances (uint32, 0xFFFFFFFF = unreachable).  weights None => unit."""
    off = _c(offsets, np.int64); idx = _c(indices, np.int32)
    w = None if weights is None else _c(weights, np.uint32)
    n = off.shape[0] - 1
    d = np.empty(n, np.uint32)
    rc = _L().oracle_dijkstra(ctypes.c_int32(n), _p(off), _p(idx), _p(w), ctypes.c_int32(source), _p(d))
    if rc and check:
        raise OracleError(rc, "dijkstra")
    return d


def bfs(offsets, indices, source: int) -> np.ndarray:
    off = _c(offsets, np.int64); idx = _c(indices, np.int32)
    n = off.shape[0] - 1
    lv = np.empty(n, np.uint32)
    rc = _L().oracle_bfs(ctypes.c_int32(n), _p(off), _p(idx), ctypes.c_int32(source), _p(lv))
    if rc:
        raise OracleError(rc, "bfs")
    return lv


def csr_transpose(offsets, indices, weights=None):
    """In-arc CSR by a stable counting sort on the target.  Returns (in_offsets int64, in_indices
    int32, in_weights uint32 or None); row v lists the sources of the arcs into v in arc order."""
    off = _c(offsets, np.int64); idx = _c(indices, np.int32)
    n = off.shape[0] - 1
    w = None if weights is None else _c(weights, np.uint32)
    ioff = np.empty(n + 1, np.int64)
    iidx = np.empty(idx.shape[0], np.int32)
    iw = None if w is None else np.empty(idx.shape[0], np.uint32)
    rc = _L().oracle_csr_transpose(ctypes.c_int32(n), _p(off), _p(idx), _p(w), _p(ioff), _p(iidx), _p(iw))
    if rc:
        raise OracleError(rc, "csr_transpose")
    return ioff, iidx, iw


def stable_marriage(men_pref, women_rank):
    """Man-proposing Gale-Shapley.  Returns (wife[m], husband[w], next[m], proposals)."""
    mp = _c(men_pref, np.int32); wr = _c(women_rank, np.int32)
    n = mp.shape[0]
    wife = np.empty(n, np.int32); hus = np.empty(n, np.int32); nxt = np.empty(n, np.int32)
    props = ctypes.c_int64(0)
    rc = _L().oracle_gale_shapley(ctypes.c_int32(n), _p(mp), _p(wr), _p(wife), _p(hus), _p(nxt),
                                  ctypes.byref(props))
    if rc:
        raise OracleError(rc, "gale_shapley")
    return wife, hus, nxt, int(props.value)


def knapsack(w, v, W: int):
    """0-1 knapsack DP.  Returns (best, final_row int32[W+1])."""
    w = _c(w, np.int32); v = _c(v, np.int32)
    row = np.empty(W + 1, np.int32)
    best = ctypes.c_int32(0)
    rc = _L().oracle_knapsack(ctypes.c_int32(w.shape[0]), _p(w), _p(v), ctypes.c_int32(W), ctypes.byref(best),
                              _p(row))
    if rc:
        raise OracleError(rc, "knapsack")
    return int(best.value), row


def transitive_closure(offsets, indices) -> np.ndarray:
    """Warshall; returns uint32[n, ceil(n/32)] bit rows (LSB-first)."""
    off = _c(offsets, np.int64); idx = _c(indices, np.int32)
    n = off.shape[0] - 1
    R = np.empty((n, (n + 31) // 32), np.uint32)
    rc = _L().oracle_warshall(ctypes.c_int32(n), _p(off), _p(idx), _p(R))
    if rc:
        raise OracleError(rc, "warshall")
    return R


def job_schedule(duration, succ_offsets, succ_indices) -> np.ndarray:
    """Topological longest path: completion times int32[n]."""
    t = _c(duration, np.int32); off = _c(succ_offsets, np.int64); idx = _c(succ_indices, np.int32)
    n = t.shape[0]
    c = np.empty(n, np.int32)
    rc = _L().oracle_job_schedule(ctypes.c_int32(n), _p(t), _p(off), _p(idx), _p(c))
    if rc:
        raise OracleError(rc, "job_schedule")
    return c


def reduce_sum(x) -> int:
    x = _c(x, np.uint64)
    return int(_L().oracle_sum_u64(ctypes.c_int64(x.shape[0]), _p(x)))
