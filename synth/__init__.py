"""Seeded synthetic inputs for the LLP problems (shared by the oracle and the CUDA path).

Nothing here computes any part of the method: the module draws random instances
and lays them out (CSR by a stable counting sort).  The C source ``gen.c`` names
the published generators it uses (SplitMix64, xoshiro256**, Lemire's bounded
integers, Knuth's Poisson).  Host arrays are numpy; the caller moves them to the
device.

Workload recipes (all seeded, all integer):

* ``er_graph``      Erdos-Renyi G(n, M) with i.i.d. ordered pairs, weights U[lo,hi].
* ``rmat_graph``    R-MAT (a, b, c, d) with a seeded vertex relabelling, weights U[lo,hi].
* ``grid_graph``    2-D 4-neighbour grid, both arc directions, independent weights.
* ``random_dag``    arcs i->j (i<j) with probability p (closure workload).
* ``job_dag``       Poisson(lambda) forward out-degree, durations U[tlo,thi].
* ``marriage``      uniform random preference permutations, or one shared men's order.
* ``knapsack``      weights U[1, W/4], values U[1, 1000].
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_SO = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into libsynth.so (host code, gcc)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O3", "-march=x86-64-v2", "-fopenmp", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = ctypes.CDLL(_SO)
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


I32, I64, U32, U64, F64 = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64,
                           ctypes.c_double)


class Csr(dict):
    """Host CSR: n, m, offsets (int64[n+1]), indices (int32[m]), weights (uint32[m] or None)."""

    @property
    def n(self):
        return self["n"]

    @property
    def m(self):
        return self["m"]


def _csr(n: int, src, dst, w) -> Csr:
    m = int(src.shape[0])
    off = np.empty(n + 1, np.int64)
    idx = np.empty(m, np.int32)
    wt = np.empty(m, np.uint32) if w is not None else None
    L = _L()
    L.synth_csr_from_edges(I32(n), I64(m), _p(src), _p(dst), _p(w) if w is not None else None,
                           _p(off), _p(idx), _p(wt) if wt is not None else None)
    return Csr(n=n, m=m, offsets=off, indices=idx, weights=wt)


def er_graph(n: int, m: int, wlo: int = 1, whi: int = 100, seed: int = 1) -> Csr:
    src = np.empty(m, np.int32); dst = np.empty(m, np.int32); w = np.empty(m, np.uint32)
    _L().synth_er_edges(I32(n), I64(m), U32(wlo), U32(whi), U64(seed), _p(src), _p(dst), _p(w))
    return _csr(n, src, dst, w)


def rmat_graph(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
               wlo: int = 1, whi: int = 255, seed: int = 2) -> Csr:
    n = 1 << scale
    m = edge_factor * n
    src = np.empty(m, np.int32); dst = np.empty(m, np.int32); w = np.empty(m, np.uint32)
    _L().synth_rmat_edges(I32(scale), I64(m), F64(a), F64(b), F64(c), U32(wlo), U32(whi), U64(seed),
                          _p(src), _p(dst), _p(w))
    g = _csr(n, src, dst, w)
    del src, dst, w
    return g


def grid_graph(rows: int, cols: int, wlo: int = 1, whi: int = 1000, seed: int = 6) -> Csr:
    cap = 4 * rows * cols
    src = np.empty(cap, np.int32); dst = np.empty(cap, np.int32); w = np.empty(cap, np.uint32)
    f = _L().synth_grid_edges
    f.restype = I64
    m = int(f(I32(rows), I32(cols), U32(wlo), U32(whi), U64(seed),
                                  _p(src), _p(dst), _p(w)))
    return _csr(rows * cols, src[:m].copy(), dst[:m].copy(), w[:m].copy())


def random_dag(n: int, pnum: int = 4, pden: int | None = None, seed: int = 6) -> Csr:
    """Arcs i->j for i<j, each with probability pnum/pden (default 4/n); no weights."""
    pden = n if pden is None else pden
    cap = max(1024, int(3 * n * pnum * (n / pden) / 2) + 64 * n)
    src = np.empty(cap, np.int32); dst = np.empty(cap, np.int32)
    f = _L().synth_random_dag_edges
    f.restype = I64
    m = int(f(I32(n), U64(pnum), U64(pden), U64(seed), I64(cap), _p(src), _p(dst)))
    if m < 0:
        raise RuntimeError("random_dag: edge buffer too small")
    return _csr(n, src[:m].copy(), dst[:m].copy(), None)


def job_dag(n: int, lam: float = 3.0, tlo: int = 1, thi: int = 100, seed: int = 5):
    """Returns (csr of successor arcs, durations int32[n])."""
    cap = 8 * n + 64
    src = np.empty(cap, np.int32); dst = np.empty(cap, np.int32); dur = np.empty(n, np.int32)
    f = _L().synth_job_dag
    f.restype = I64
    m = int(f(I32(n), F64(lam), I32(tlo), I32(thi), U64(seed), I64(cap), _p(src), _p(dst), _p(dur)))
    if m < 0:
        raise RuntimeError("job_dag: edge buffer too small")
    return _csr(n, src[:m].copy(), dst[:m].copy(), None), dur


def marriage(n: int, seed: int = 3, adversarial: bool = False):
    """Returns (men_pref int32[n,n], women_rank int32[n,n])."""
    mp = np.empty((n, n), np.int32); wr = np.empty((n, n), np.int32)
    _L().synth_marriage(I32(n), U64(seed), ctypes.c_int(1 if adversarial else 0), _p(mp), _p(wr))
    return mp, wr


def knapsack(n: int, W: int, seed: int = 5, stream: int = 0, vlo: int = 1, vhi: int = 1000):
    """Returns (weights int32[n] in [1, max(1, W//4)], values int32[n] in [vlo, vhi])."""
    w = np.empty(n, np.int32); v = np.empty(n, np.int32)
    _L().synth_knapsack(I32(n), I32(W), I32(vlo), I32(vhi), U64(seed), U64(stream), _p(w), _p(v))
    return w, v


def u64(n: int, seed: int = 7) -> np.ndarray:
    x = np.empty(n, np.uint64)
    _L().synth_fill_u64(I64(n), U64(seed), _p(x))
    return x


def i32(n: int, lo: int, hi: int, seed: int, stream: int = 0) -> np.ndarray:
    x = np.empty(n, np.int32)
    _L().synth_fill_i32(I64(n), I32(lo), I32(hi), U64(seed), U64(stream), _p(x))
    return x


def sizes(count: int, lo: int, hi: int, seed: int, stream: int) -> np.ndarray:
    x = np.empty(count, np.int64)
    _L().synth_sizes(I32(count), I64(lo), I64(hi), U64(seed), U64(stream), _p(x))
    return x


def max_out_degree_vertex(g: Csr) -> int:
    """Highest out-degree vertex, ties to the smallest id."""
    return int(np.argmax(np.diff(g["offsets"])))


# ------------------------------------------------------------ named workloads

def er16k(seed: int = 1) -> Csr:
    """16,384 vertices, 131,072 i.i.d. arcs, weights U[1,100]; source 0."""
    return er_graph(16384, 131072, 1, 100, seed)


def rmat(scale: int = 22, seed: int = 2) -> Csr:
    """R-MAT scale `scale`, edge factor 16, (.57,.19,.19,.05), weights U[1,255]."""
    return rmat_graph(scale, 16, 0.57, 0.19, 0.19, 1, 255, seed)


def knapsack_batch(count: int = 4096, nlo: int = 16, nhi: int = 2048, Wlo: int = 256, Whi: int = 65536,
                   seed: int = 5):
    """Batch of 0-1 knapsack instances, concatenated: item_off int64[count+1], w, v, capacity."""
    ns = sizes(count, nlo, nhi, seed, 101)
    Ws = sizes(count, Wlo, Whi, seed, 102)
    off = np.zeros(count + 1, np.int64)
    off[1:] = np.cumsum(ns)
    w = np.empty(int(off[-1]), np.int32); v = np.empty(int(off[-1]), np.int32)
    for i in range(count):
        wi, vi = knapsack(int(ns[i]), int(Ws[i]), seed, 1000 + i)
        w[off[i]:off[i + 1]] = wi
        v[off[i]:off[i + 1]] = vi
    return dict(count=count, item_off=off, w=w, v=v, capacity=Ws.astype(np.int32))


def job_batch(count: int = 2048, nlo: int = 64, nhi: int = 8192, seed: int = 5):
    """Batch of job DAGs, concatenated with local (per-DAG) vertex ids."""
    ns = sizes(count, nlo, nhi, seed, 201)
    job_off = np.zeros(count + 1, np.int64); job_off[1:] = np.cumsum(ns)
    offs, idxs, durs, edge_off = [], [], [], [0]
    for i in range(count):
        g, d = job_dag(int(ns[i]), 3.0, 1, 100, seed * 1000003 + i)
        offs.append(g["offsets"][:-1] + edge_off[-1]); idxs.append(g["indices"]); durs.append(d)
        edge_off.append(edge_off[-1] + g["m"])
    offsets = np.concatenate(offs + [np.array([edge_off[-1]], np.int64)])
    return dict(count=count, job_off=job_off, edge_off=np.array(edge_off, np.int64),
                succ_offsets=offsets, succ_indices=np.concatenate(idxs), duration=np.concatenate(durs))


def marriage_batch(count: int = 1024, nlo: int = 32, nhi: int = 1024, seed: int = 5):
    """Batch of random stable-marriage instances; pref_off[i] = start of instance i's n_i*n_i block."""
    ns = sizes(count, nlo, nhi, seed, 301).astype(np.int32)
    sq = ns.astype(np.int64) ** 2
    pref_off = np.zeros(count + 1, np.int64); pref_off[1:] = np.cumsum(sq)
    mp = np.empty(int(pref_off[-1]), np.int32); wr = np.empty(int(pref_off[-1]), np.int32)
    for i in range(count):
        a, b = marriage(int(ns[i]), seed * 1000003 + 7 * i + 1)
        mp[pref_off[i]:pref_off[i + 1]] = a.ravel(); wr[pref_off[i]:pref_off[i + 1]] = b.ravel()
    return dict(count=count, n=ns, pref_off=pref_off, men_pref=mp, women_rank=wr)


def graph_batch(count: int = 2048, nlo: int = 64, nhi: int = 8192, seed: int = 5, bfs_every: int = 4):
    """Batch of small graphs for batched SSSP/BFS, concatenated with local vertex ids.
    Instance i is, by i mod 4: uniform (ER, n ~ U[nlo, nhi], 2-12 arcs per vertex, weights
    U[1,255]), R-MAT (power law, scale from the drawn n, edge factor 8, weights U[1,255]),
    a 4-neighbour grid (road-like, side from the drawn n, weights U[1,1000]), or uniform
    again; sources: vertex 0, or the highest out-degree vertex for R-MAT.  Every bfs_every-th
    instance is a BFS (unit = 1)."""
    ns = sizes(count, nlo, nhi, seed, 401)
    degs = sizes(count, 2, 12, seed, 402)
    verts, arc_off, idxs, ws, srcs = [0], [], [], [], []
    base = 0
    for i in range(count):
        n, s = int(ns[i]), seed * 1000003 + 11 * i + 3
        kind = i % 4
        if kind == 1:
            g = rmat_graph(max(1, int(n).bit_length() - 1), 8, 0.57, 0.19, 0.19, 1, 255, seed=s)
            src = max_out_degree_vertex(g)
        elif kind == 2:
            side = max(2, int(np.sqrt(n)))
            g = grid_graph(side, side, 1, 1000, seed=s)
            src = 0
        else:
            g = er_graph(n, n * int(degs[i]), 1, 255, seed=s)
            src = 0
        arc_off.append(g["offsets"][:-1] + base)
        idxs.append(g["indices"]); ws.append(g["weights"]); srcs.append(src)
        base += g["m"]
        verts.append(verts[-1] + g["n"])
    unit = np.array([1 if bfs_every and i % bfs_every == bfs_every - 1 else 0 for i in range(count)], np.int32)
    return dict(count=count, off=np.array(verts, np.int64),
                arc_offsets=np.concatenate(arc_off + [np.array([base], np.int64)]),
                indices=np.concatenate(idxs), weights=np.concatenate(ws), source=np.array(srcs, np.int32),
                unit=unit)
