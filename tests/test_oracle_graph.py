"""Pins of the SSSP, BFS and closure oracles against the paper and the mathematics."""
import itertools

import numpy as np
import pytest

import oracle
import synth
from conftest import read_golden

INF = oracle.INF


def csr_from_arcs(n, arcs, with_w=True):
    arcs = sorted(enumerate(arcs), key=lambda t: (t[1][0], t[0]))
    off = np.zeros(n + 1, np.int64)
    for _, a in arcs:
        off[a[0] + 1] += 1
    off = np.cumsum(off)
    idx = np.array([a[1] for _, a in arcs], np.int32)
    w = np.array([a[2] for _, a in arcs], np.uint32) if with_w else None
    return off, idx, w


def brute_sssp(n, arcs, s):
    """Minimum over all simple paths from s (explicit enumeration, tiny n)."""
    best = [None] * n
    best[s] = 0
    adj = {}
    for u, v, w in arcs:
        adj.setdefault(u, []).append((v, w))

    def dfs(u, dist, seen):
        for v, w in adj.get(u, []):
            if v in seen:
                continue
            nd = dist + w
            if best[v] is None or nd < best[v]:
                best[v] = nd
            dfs(v, nd, seen | {v})

    dfs(s, 0, {s})
    return np.array([INF if b is None else b for b in best], np.uint32)


def random_arcs(rng, n, m, wmax):
    return [(int(rng.integers(n)), int(rng.integers(n)), int(rng.integers(1, wmax + 1))) for _ in range(m)]


def test_sssp_paper_example():
    g = read_golden("sssp_paper_example.txt")
    n = int(g["n"][0])
    arcs = [tuple(int(x) for x in a.split()) for a in g["arc"]]
    off, idx, w = csr_from_arcs(n, arcs)
    d = oracle.sssp(off, idx, w, int(g["source"][0]))
    assert d.tolist() == [int(x) for x in g["final"][0].split()]
    assert d[3] == int(g["race_correct_d3"][0])


def test_sssp_chain_is_linear():
    n = 1000
    arcs = [(i, i + 1, 1) for i in range(n - 1)]
    off, idx, w = csr_from_arcs(n, arcs)
    assert (oracle.sssp(off, idx, w, 0) == np.arange(n)).all()
    # source in the middle: vertices before it are unreachable
    d = oracle.sssp(off, idx, w, 500)
    assert (d[:500] == INF).all() and (d[500:] == np.arange(500)).all()


@pytest.mark.parametrize("seed", range(40))
def test_sssp_brute_force_tiny(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 9))
    arcs = random_arcs(rng, n, int(rng.integers(0, 20)), 9)
    off, idx, w = csr_from_arcs(n, arcs)
    s = int(rng.integers(n))
    assert (oracle.sssp(off, idx, w, s) == brute_sssp(n, arcs, s)).all()


def bellman_ford(n, arcs, s):
    d = [None] * n
    d[s] = 0
    for _ in range(n):
        for u, v, w in arcs:
            if d[u] is not None and (d[v] is None or d[u] + w < d[v]):
                d[v] = d[u] + w
    return np.array([INF if x is None else x for x in d], np.uint32)


@pytest.mark.parametrize("seed", range(5))
def test_sssp_matches_bellman_ford(seed):
    rng = np.random.default_rng(100 + seed)
    n = 60
    arcs = random_arcs(rng, n, 240, 50)
    off, idx, w = csr_from_arcs(n, arcs)
    assert (oracle.sssp(off, idx, w, 0) == bellman_ford(n, arcs, 0)).all()


def check_sssp_invariants(off, idx, w, s, d):
    """d[s]=0; d[v] <= d[u]+w(u,v) on every arc; every reached v != s has a tight in-arc.
    With weights >= 1 these fix d uniquely."""
    n = off.shape[0] - 1
    src = np.repeat(np.arange(n), np.diff(off))
    du = d[src].astype(np.int64)
    dv = d[idx].astype(np.int64)
    ww = np.ones(idx.shape[0], np.int64) if w is None else w.astype(np.int64)
    reached_u = d[src] != INF
    assert d[s] == 0
    assert (dv[reached_u] <= du[reached_u] + ww[reached_u]).all()
    tight = np.zeros(n, bool)
    t = reached_u & (dv == du + ww)
    tight[idx[t]] = True
    reached = d != INF
    reached[s] = False
    assert tight[reached].all()


def test_sssp_invariants_er():
    g = synth.er_graph(3000, 20000, 1, 100, seed=9)
    d = oracle.sssp(g["offsets"], g["indices"], g["weights"], 0)
    check_sssp_invariants(g["offsets"], g["indices"], g["weights"], 0, d)
    assert (d != INF).sum() > 2000


def test_sssp_overflow_reported():
    arcs = [(0, 1, 0xF0000000), (1, 2, 0xF0000000)]
    off, idx, w = csr_from_arcs(3, arcs)
    with pytest.raises(oracle.OracleError) as e:
        oracle.sssp(off, idx, w, 0)
    assert e.value.code == oracle.ERR_OVERFLOW


def test_bfs_paper_race_example():
    g = read_golden("bfs_race_example.txt")
    n = int(g["n"][0])
    arcs = [tuple(int(x) for x in a.split()) + (1,) for a in g["arc"]]
    off, idx, _ = csr_from_arcs(n, arcs)
    assert oracle.bfs(off, idx, 0).tolist() == [int(x) for x in g["level"][0].split()]


@pytest.mark.parametrize("seed", range(20))
def test_bfs_brute_force_tiny(seed):
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(1, 9))
    arcs = [(a, b, 1) for a, b, _ in random_arcs(rng, n, int(rng.integers(0, 16)), 1)]
    off, idx, _ = csr_from_arcs(n, arcs)
    assert (oracle.bfs(off, idx, 0) == brute_sssp(n, arcs, 0)).all()


def test_bfs_is_unit_weight_sssp():
    g = synth.rmat_graph(12, 8, seed=3)
    s = synth.max_out_degree_vertex(g)
    lv = oracle.bfs(g["offsets"], g["indices"], s)
    assert (lv == oracle.sssp(g["offsets"], g["indices"], None, s)).all()
    check_sssp_invariants(g["offsets"], g["indices"], None, s, lv)


# ---------------------------------------------------------------- closure

def closure_dfs(n, arcs):
    adj = [[] for _ in range(n)]
    for u, v in arcs:
        adj[u].append(v)
    R = np.zeros((n, n), bool)
    for s in range(n):
        stack = list(adj[s])
        while stack:
            v = stack.pop()
            if not R[s, v]:
                R[s, v] = True
                stack.extend(adj[v])
    return R


def unpack(Rb, n):
    bits = np.unpackbits(Rb.view(np.uint8), axis=1, bitorder="little")
    return bits[:, :n].astype(bool)


@pytest.mark.parametrize("seed", range(30))
def test_closure_matches_dfs(seed):
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(1, 9)) if seed < 20 else int(rng.integers(30, 80))
    m = int(rng.integers(0, 3 * n + 1))
    arcs = [(int(rng.integers(n)), int(rng.integers(n))) for _ in range(m)]  # cycles allowed
    off, idx, _ = csr_from_arcs(n, [(a, b, 1) for a, b in arcs])
    R = unpack(oracle.transitive_closure(off, idx), n)
    assert (R == closure_dfs(n, arcs)).all()


def test_closure_idempotent_and_transitive():
    g = synth.random_dag(300, 4, seed=5)
    n = g.n
    R = unpack(oracle.transitive_closure(g["offsets"], g["indices"]), n)
    # R contains the adjacency
    src = np.repeat(np.arange(n), np.diff(g["offsets"]))
    assert R[src, g["indices"]].all()
    # closure of the closure graph is itself
    u, v = np.nonzero(R)
    off, idx, _ = csr_from_arcs(n, list(zip(u.tolist(), v.tolist(), [1] * len(u))))
    R2 = unpack(oracle.transitive_closure(off, idx), n)
    assert (R2 == R).all()
    # transitive: R @ R subset of R; irreflexive on a DAG
    RR = (R.astype(np.int32) @ R.astype(np.int32)) > 0
    assert not (RR & ~R).any()
    assert not np.diag(R).any()


def test_closure_chain_closed_form():
    n = 70
    off, idx, _ = csr_from_arcs(n, [(i, i + 1, 1) for i in range(n - 1)])
    R = unpack(oracle.transitive_closure(off, idx), n)
    assert (R == np.triu(np.ones((n, n), bool), 1)).all()


# -------------------------------------------------------------- transpose

@pytest.mark.parametrize("seed", range(10))
def test_transpose_brute_force_tiny(seed):
    """Row v of the in-arc CSR = the (source, weight) of every arc into v, in arc order."""
    rng = np.random.default_rng(700 + seed)
    n = int(rng.integers(1, 9))
    arcs = random_arcs(rng, n, int(rng.integers(0, 25)), 9)
    off, idx, w = csr_from_arcs(n, arcs)
    ioff, iidx, iw = oracle.csr_transpose(off, idx, w)
    src = np.repeat(np.arange(n), np.diff(off))
    for v in range(n):
        want = [(int(src[e]), int(w[e])) for e in range(len(idx)) if idx[e] == v]
        got = list(zip(iidx[ioff[v]:ioff[v + 1]].tolist(), iw[ioff[v]:ioff[v + 1]].tolist()))
        assert got == want
    assert ioff[0] == 0 and ioff[-1] == len(idx)


def test_transpose_twice_sorts_rows():
    """T(T(g)) is g with each row stably sorted by target."""
    g = synth.rmat_graph(10, 8, seed=5)
    ioff, iidx, iw = oracle.csr_transpose(g["offsets"], g["indices"], g["weights"])
    off2, idx2, w2 = oracle.csr_transpose(ioff, iidx, iw)
    assert (off2 == g["offsets"]).all()
    for u in range(g["n"]):
        a, b = g["offsets"][u], g["offsets"][u + 1]
        order = np.argsort(g["indices"][a:b], kind="stable")
        assert (idx2[a:b] == g["indices"][a:b][order]).all()
        assert (w2[a:b] == g["weights"][a:b][order]).all()


def test_transpose_reverses_reachability():
    """v is reachable from s in g iff s is reachable from v in the transpose."""
    rng = np.random.default_rng(9)
    n = 60
    off, idx, _ = csr_from_arcs(n, random_arcs(rng, n, 90, 1), with_w=False)
    ioff, iidx, _ = oracle.csr_transpose(off, idx)
    fwd = np.stack([oracle.bfs(off, idx, s) != INF for s in range(n)])
    bwd = np.stack([oracle.bfs(ioff, iidx, v) != INF for v in range(n)])
    assert (fwd == bwd.T).all()
    lv = oracle.bfs(off, idx, 0)
    # levels read through in-arcs: level(v) = 1 + min level over in-neighbours (Sec. 4.2)
    for v in range(1, n):
        ins = iidx[ioff[v]:ioff[v + 1]]
        fin = [int(lv[u]) for u in ins if lv[u] != INF]
        assert lv[v] == (min(fin) + 1 if fin else INF)
