"""GPU parity of llp_sssp / llp_bfs (through the C ABI) against the oracle, bit-exact."""
import numpy as np
import pytest

import oracle
import synth
from conftest import read_golden

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def llp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_13147_b300 as m
    m.lib()
    return m


def dev_graph(llp, g, offsets_64=False):
    return llp.DeviceGraph.from_host(g, "cuda", offsets_64=offsets_64)


def run_sssp(llp, g, s, **kw):
    dg = dev_graph(llp, g, kw.pop("offsets_64", False))
    sched = llp.make_sched(**kw) if kw else None
    d, ws = llp.sssp(dg, s, sched=sched)
    st = llp.get_status(ws)
    assert st["status"] == 0, st
    return llp.as_u32(d), st


def run_bfs(llp, g, s, **kw):
    dg = dev_graph(llp, g, kw.pop("offsets_64", False))
    sched = llp.make_sched(**kw) if kw else None
    d, ws = llp.bfs(dg, s, sched=sched)
    st = llp.get_status(ws)
    assert st["status"] == 0, st
    return llp.as_u32(d), st


def csr_from_arcs(n, arcs):
    arcs = sorted(enumerate(arcs), key=lambda t: (t[1][0], t[0]))
    off = np.zeros(n + 1, np.int64)
    for _, a in arcs:
        off[a[0] + 1] += 1
    return dict(n=n, m=len(arcs), offsets=np.cumsum(off), indices=np.array([a[1] for _, a in arcs], np.int32),
                weights=np.array([a[2] for _, a in arcs], np.uint32))


SCHEDS = [dict(), dict(mode=1), dict(mode=2), dict(mode=1, delta=64), dict(mode=0, delta=8, block_cfg=1),
          dict(mode=2, delta=300, block_cfg=3, threads=256), dict(delta=1, block_cfg=1),
          dict(mode=1, local_chain=4), dict(mode=2, local_chain=16, delta=500), dict(local_chain=64, block_cfg=3),
          dict(mode=1, local_chain=1, delta=1, threads=256),
          # dense-sweep group widths; fixed-state memoization (needs buckets); the load-balanced engine
          dict(group_words=1), dict(mode=2, group_words=2, block_cfg=1), dict(group_words=4, delta=64, fixed_memo=1),
          dict(mode=1, delta=8, fixed_memo=1), dict(mode=2, delta=300, fixed_memo=1, local_chain=4),
          dict(block_cfg=4), dict(block_cfg=4, mode=1), dict(block_cfg=4, mode=2, threads=256)]


def test_paper_example(llp):
    gd = read_golden("sssp_paper_example.txt")
    n = int(gd["n"][0])
    g = csr_from_arcs(n, [tuple(int(x) for x in a.split()) for a in gd["arc"]])
    for kw in SCHEDS:
        d, _ = run_sssp(llp, g, 0, **kw)
        assert d.tolist() == [int(x) for x in gd["final"][0].split()]


@pytest.mark.parametrize("kw", SCHEDS)
def test_sssp_er16k_all_schedules(llp, kw):
    g = synth.er16k()
    ref = oracle.sssp(g["offsets"], g["indices"], g["weights"], 0)
    d, st = run_sssp(llp, g, 0, **kw)
    assert (d == ref).all()
    assert st["advances"] >= int((ref != oracle.INF).sum()) - 1


@pytest.mark.parametrize("kw", SCHEDS[:4] + SCHEDS[7:9])
def test_bfs_er16k(llp, kw):
    g = synth.er16k()
    ref = oracle.bfs(g["offsets"], g["indices"], 0)
    d, _ = run_bfs(llp, g, 0, **kw)
    assert (d == ref).all()


def test_chain_many_sweeps(llp):
    n = 3000
    g = csr_from_arcs(n, [(i, i + 1, 1 + (i % 7)) for i in range(n - 1)])
    ref = oracle.sssp(g["offsets"], g["indices"], g["weights"], 0)
    d, st = run_sssp(llp, g, 0)
    assert (d == ref).all()
    assert st["sweeps"] >= n - 1  # one vertex becomes forbidden per sweep
    assert st["items"] == n - 1   # informed selection: O(n) work (the paper's chain claim)


@pytest.mark.parametrize("seed", range(12))
def test_random_small_and_ragged(llp, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 3000))
    m = int(rng.integers(0, 6 * n))
    arcs = [(int(rng.integers(n)), int(rng.integers(n)), int(rng.integers(1, 1000))) for _ in range(m)]
    # a few hubs to exercise the chunk path
    for h in range(min(3, n)):
        arcs += [(h, int(rng.integers(n)), int(rng.integers(1, 50))) for _ in range(int(rng.integers(0, 1500)))]
    g = csr_from_arcs(n, arcs)
    s = int(rng.integers(n))
    ref = oracle.sssp(g["offsets"], g["indices"], g["weights"], s)
    for kw in SCHEDS[::2]:
        d, _ = run_sssp(llp, g, s, offsets_64=bool(seed % 2), **kw)
        assert (d == ref).all(), kw
    refb = oracle.bfs(g["offsets"], g["indices"], s)
    d, _ = run_bfs(llp, g, s)
    assert (d == refb).all()


@pytest.mark.parametrize("kw", [dict(), dict(mode=1, local_chain=16), dict(mode=2, local_chain=4, delta=2000),
                                dict(mode=2, local_chain=4, delta=2000, fixed_memo=1), dict(delta=500, fixed_memo=1),
                                dict(block_cfg=4), dict(group_words=8)])
def test_grid_graph_schedules(llp, kw):
    """Road-like input (2-D grid, both arc directions): long paths, thousands of sweeps."""
    g = synth.grid_graph(96, 77, 1, 1000, seed=5)
    ref = oracle.sssp(g["offsets"], g["indices"], g["weights"], 5)
    d, _ = run_sssp(llp, g, 5, **kw)
    assert (d == ref).all()
    lv, _ = run_bfs(llp, g, 5, **kw)
    assert (lv == oracle.bfs(g["offsets"], g["indices"], 5)).all()


@pytest.mark.parametrize("n", [31, 33, 1023, 1025])
def test_ragged_vertex_counts(llp, n):
    """n not a multiple of the 32-vertex bitmap word; source = last vertex."""
    rng = np.random.default_rng(n)
    arcs = [(int(rng.integers(n)), int(rng.integers(n)), int(rng.integers(1, 20))) for _ in range(4 * n)]
    arcs += [(n - 1, int(rng.integers(n)), 1) for _ in range(70)]  # a large source vertex
    g = csr_from_arcs(n, arcs)
    for kw in (dict(), dict(mode=2), dict(mode=1, local_chain=4)):
        d, _ = run_sssp(llp, g, n - 1, **kw)
        assert (d == oracle.sssp(g["offsets"], g["indices"], g["weights"], n - 1)).all()


def test_edge_cases(llp):
    # single vertex, no arcs
    g = dict(n=1, m=0, offsets=np.zeros(2, np.int64), indices=np.zeros(0, np.int32), weights=np.zeros(0, np.uint32))
    d, st = run_sssp(llp, g, 0)
    assert d.tolist() == [0]
    # source without out-arcs
    g = csr_from_arcs(5, [(1, 2, 3), (2, 3, 4)])
    d, _ = run_sssp(llp, g, 0)
    assert d.tolist() == [0] + [oracle.INF] * 4
    # self loops and parallel arcs
    g = csr_from_arcs(3, [(0, 0, 1), (0, 1, 9), (0, 1, 4), (1, 1, 2), (1, 2, 7), (1, 2, 5)])
    d, _ = run_sssp(llp, g, 0)
    assert d.tolist() == [0, 4, 9]


def test_overflow_is_reported(llp):
    g = csr_from_arcs(3, [(0, 1, 0xF0000000), (1, 2, 0xF0000000)])
    dg = dev_graph(llp, g)
    _, ws = llp.sssp(dg, 0)
    assert llp.get_status(ws)["status"] == llp.LLP_ERR_OVERFLOW


def test_deadline_returns_timeout_and_context_survives(llp):
    """A wait limit that runs out ends the kernel with LLP_ERR_TIMEOUT (no fault);
    the next call on the same workspace is correct."""
    n = 20000
    g = csr_from_arcs(n, [(i, i + 1, 1) for i in range(n - 1)])
    dg = dev_graph(llp, g)
    _, ws = llp.sssp(dg, 0, sched=llp.make_sched(deadline_ns=1))
    assert llp.get_status(ws)["status"] == llp.LLP_ERR_TIMEOUT
    d, ws = llp.sssp(dg, 0, ws=ws)
    assert llp.get_status(ws)["status"] == 0
    assert (llp.as_u32(d) == np.arange(n)).all()


@pytest.mark.parametrize("kw", SCHEDS)
def test_rmat16_schedules(llp, kw):
    g = synth.rmat(16, seed=21)
    s = synth.max_out_degree_vertex(g)
    ref = oracle.sssp(g["offsets"], g["indices"], g["weights"], s)
    d, _ = run_sssp(llp, g, s, **kw)
    assert (d == ref).all()


@pytest.fixture(scope="module")
def rmat22():
    return synth.rmat(22)


def test_rmat22_sssp_full(llp, rmat22):
    """Full-size R-MAT scale 22 (67,108,864 arcs), default schedule as benchmarked."""
    g = rmat22
    s = synth.max_out_degree_vertex(g)
    ref = oracle.sssp(g["offsets"], g["indices"], g["weights"], s)
    d, st = run_sssp(llp, g, s)
    assert (d == ref).all()
    # the load-balanced engine and fixed-state memoization (with buckets) on the same graph
    for kw in (dict(block_cfg=4), dict(delta=512, fixed_memo=1)):
        d, _ = run_sssp(llp, g, s, **kw)
        assert (d == ref).all(), kw


def test_rmat22_bfs_full(llp, rmat22):
    g = rmat22
    s = synth.max_out_degree_vertex(g)
    ref = oracle.bfs(g["offsets"], g["indices"], s)
    d, _ = run_bfs(llp, g, s)
    assert (d == ref).all()
    d64, _ = run_bfs(llp, g, s, offsets_64=True)
    assert (d64 == ref).all()


# ----------------------------------------------- BFS with pull sweeps (in-arcs)

def run_bfs_pull(llp, g, s, **kw):
    dg = dev_graph(llp, g, kw.pop("offsets_64", False))
    gt = dg.transpose()
    sched = llp.make_sched(**kw) if kw else None
    d, ws = llp.bfs_pull(dg, gt, s, sched=sched)
    st = llp.get_status(ws)
    assert st["status"] == 0, st
    return llp.as_u32(d), st


def check_transpose(llp, g, offsets_64):
    dg = dev_graph(llp, g, offsets_64)
    gt = dg.transpose(with_weights=g.get("weights") is not None)
    ws = gt.transpose_ws
    assert llp.get_status(ws)["status"] == 0
    ioff, iidx, iw = oracle.csr_transpose(g["offsets"], g["indices"], g.get("weights"))
    off = gt.offsets.cpu().numpy()
    assert off.dtype == (np.int64 if offsets_64 else np.int32)
    assert (off.astype(np.int64) == ioff).all()
    idx = gt.indices.cpu().numpy()
    w = gt.weights.cpu().numpy().view(np.uint32) if gt.weights is not None else np.zeros_like(idx)
    rw = iw if iw is not None else np.zeros_like(iidx)
    # rows as multisets of (source, weight): the order within a row is unspecified
    row = np.repeat(np.arange(g["n"]), np.diff(ioff))
    a = np.lexsort((w.astype(np.int64), idx, row))
    b = np.lexsort((rw.astype(np.int64), iidx, row))
    assert (idx[a] == iidx[b]).all() and (w[a] == rw[b]).all()


@pytest.mark.parametrize("seed", range(6))
def test_transpose_matches_oracle(llp, seed):
    rng = np.random.default_rng(400 + seed)
    n = int(rng.integers(1, 5000))
    arcs = [(int(rng.integers(n)), int(rng.integers(n)), int(rng.integers(1, 1000)))
            for _ in range(int(rng.integers(0, 8 * n)))]
    arcs += [(int(rng.integers(n)), 0, 7) for _ in range(int(rng.integers(0, 3000)))]  # a high in-degree target
    check_transpose(llp, csr_from_arcs(n, arcs), bool(seed % 2))


def test_transpose_rmat16(llp):
    check_transpose(llp, synth.rmat(16, seed=21), False)


PULL_SCHEDS = [dict(), dict(pull_permille=1), dict(pull_permille=-1), dict(pull_permille=1, mode=2),
               dict(pull_permille=1, block_cfg=1), dict(pull_permille=5, block_cfg=3, threads=256),
               dict(pull_permille=1, mode=1, block_cfg=3), dict(pull_permille=1, local_chain=4)]


@pytest.mark.parametrize("kw", PULL_SCHEDS)
def test_bfs_pull_er16k(llp, kw):
    g = synth.er16k()
    d, st = run_bfs_pull(llp, g, 0, **kw)
    assert (d == oracle.bfs(g["offsets"], g["indices"], 0)).all()
    if kw.get("pull_permille") == 1 and not kw.get("local_chain"):
        # every sweep pulls except the first (the source alone is below m / 1000 arcs) and the
        # last (empty frontier)
        assert st["pull_sweeps"] == st["sweeps"] - 2 > 0
    if kw.get("pull_permille") == -1 or kw.get("local_chain"):
        assert st["pull_sweeps"] == 0


@pytest.mark.parametrize("seed", range(8))
def test_bfs_pull_random_ragged(llp, seed):
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(1, 4000))
    arcs = [(int(rng.integers(n)), int(rng.integers(n)), 1) for _ in range(int(rng.integers(0, 6 * n)))]
    for h in range(min(3, n)):  # hubs: large out-degree and large in-degree
        arcs += [(h, int(rng.integers(n)), 1) for _ in range(int(rng.integers(0, 1500)))]
        arcs += [(int(rng.integers(n)), n - 1 - h, 1) for _ in range(int(rng.integers(0, 1500)))]
    g = csr_from_arcs(n, arcs)
    s = int(rng.integers(n))
    ref = oracle.bfs(g["offsets"], g["indices"], s)
    for kw in (dict(), dict(pull_permille=1), dict(pull_permille=20, block_cfg=1)):
        d, _ = run_bfs_pull(llp, g, s, offsets_64=bool(seed % 2), **kw)
        assert (d == ref).all(), kw


def test_bfs_pull_push_pull_alternation(llp):
    """Wide, narrow, wide frontiers: pull, push, pull.  The push sweep between them reaches
    vertices (a ring) that the second pull sweep must see as reached."""
    L = 1000
    X = L + 1
    arcs = [(0, 1 + i, 1) for i in range(L)] + [(1 + i, X, 1) for i in range(L)]
    arcs += [(X, X + 1 + i, 1) for i in range(L)]
    arcs += [(X + 1 + i, X + 1 + (i + 1) % L, 1) for i in range(L)]
    arcs += [(X + 1 + i, X + 1 + L + i, 1) for i in range(L)]
    n = X + 1 + 2 * L
    g = csr_from_arcs(n, arcs)
    d, st = run_bfs_pull(llp, g, 0, pull_permille=300)
    assert (d == oracle.bfs(g["offsets"], g["indices"], 0)).all()
    assert st["pull_sweeps"] == 2
    assert d[X] == 2 and d[X + 1] == 3 and d[n - 1] == 4


@pytest.mark.parametrize("kw", [dict(), dict(pull_permille=1)])
def test_bfs_pull_grid(llp, kw):
    g = synth.grid_graph(96, 77, 1, 1000, seed=5)
    d, _ = run_bfs_pull(llp, g, 5, **kw)
    assert (d == oracle.bfs(g["offsets"], g["indices"], 5)).all()


@pytest.mark.parametrize("n", [31, 33, 1023, 1025])
def test_bfs_pull_ragged_vertex_counts(llp, n):
    rng = np.random.default_rng(n + 1)
    arcs = [(int(rng.integers(n)), int(rng.integers(n)), 1) for _ in range(4 * n)]
    arcs += [(n - 1, int(rng.integers(n)), 1) for _ in range(70)]
    g = csr_from_arcs(n, arcs)
    for kw in (dict(pull_permille=1), dict()):
        d, _ = run_bfs_pull(llp, g, n - 1, **kw)
        assert (d == oracle.bfs(g["offsets"], g["indices"], n - 1)).all()


def test_bfs_pull_edge_cases(llp):
    g = dict(n=1, m=0, offsets=np.zeros(2, np.int64), indices=np.zeros(0, np.int32), weights=None)
    d, _ = run_bfs_pull(llp, g, 0, pull_permille=1)
    assert d.tolist() == [0]
    g = csr_from_arcs(5, [(1, 2, 1), (2, 3, 1)])  # source without out-arcs
    d, _ = run_bfs_pull(llp, g, 0, pull_permille=1)
    assert d.tolist() == [0] + [oracle.INF] * 4
    g = csr_from_arcs(3, [(0, 0, 1), (0, 1, 1), (0, 1, 1), (1, 1, 1), (1, 2, 1), (1, 2, 1)])
    d, _ = run_bfs_pull(llp, g, 0, pull_permille=1)
    assert d.tolist() == [0, 1, 2]


@pytest.mark.parametrize("kw", [dict(), dict(pull_permille=10), dict(pull_permille=200, block_cfg=3)])
def test_bfs_pull_rmat16(llp, kw):
    g = synth.rmat(16, seed=21)
    s = synth.max_out_degree_vertex(g)
    d, st = run_bfs_pull(llp, g, s, **kw)
    assert (d == oracle.bfs(g["offsets"], g["indices"], s)).all()
    assert st["pull_sweeps"] >= 1


def test_rmat22_bfs_pull_full(llp, rmat22):
    """Full-size R-MAT scale 22 with its device transpose, default schedule as benchmarked."""
    g = rmat22
    s = synth.max_out_degree_vertex(g)
    ref = oracle.bfs(g["offsets"], g["indices"], s)
    d, st = run_bfs_pull(llp, g, s)
    assert (d == ref).all()
    assert st["pull_sweeps"] >= 1
    d64, _ = run_bfs_pull(llp, g, s, offsets_64=True)
    assert (d64 == ref).all()


# ------------------------------------------------- warm start (incremental re-solve)

def shorten(g, rng, frac_dec, n_ins, wmax=100):
    """Decrease a random fraction of the weights and insert random arcs.  Returns the new graph
    (CSR, arcs sorted by tail) and the tails of every changed or inserted arc."""
    n = g["n"]
    src = np.repeat(np.arange(n, dtype=np.int32), np.diff(g["offsets"]))
    dst = g["indices"].copy()
    w = g["weights"].copy()
    dec = rng.random(len(w)) < frac_dec
    w[dec] = np.maximum(1, w[dec] // 3)
    ins_s = rng.integers(0, n, n_ins).astype(np.int32)
    ins_d = rng.integers(0, n, n_ins).astype(np.int32)
    ins_w = rng.integers(1, wmax + 1, n_ins).astype(np.uint32)
    src = np.concatenate([src, ins_s]); dst = np.concatenate([dst, ins_d]); w = np.concatenate([w, ins_w])
    order = np.argsort(src, kind="stable")
    off = np.zeros(n + 1, np.int64)
    np.add.at(off, src + 1, 1)
    gn = dict(n=n, m=len(dst), offsets=np.cumsum(off), indices=dst[order], weights=w[order])
    seeds = np.unique(np.concatenate([src[:len(dec)][dec], ins_s])).astype(np.int32)
    return gn, seeds


def run_warm(llp, g, s, d_old, seeds, unit=False, **kw):
    dg = dev_graph(llp, g, kw.pop("offsets_64", False))
    sched = llp.make_sched(**kw) if kw else None
    dist = torch.from_numpy(d_old.view(np.int32).copy()).cuda()
    sd = torch.from_numpy(seeds).cuda() if seeds is not None and len(seeds) else None
    f = llp.bfs_warm if unit else llp.sssp_warm
    d, ws = f(dg, s, dist, sd, sched=sched)
    st = llp.get_status(ws)
    assert st["status"] == 0, st
    return llp.as_u32(d), st


@pytest.mark.parametrize("kw", [dict(), dict(mode=1, delta=64), dict(mode=2), dict(mode=1, local_chain=16),
                                dict(delta=300, block_cfg=3, threads=256), dict(block_cfg=4),
                                dict(block_cfg=4, mode=2), dict(delta=64, fixed_memo=1)])
def test_warm_er16k(llp, kw):
    g = synth.er16k()
    rng = np.random.default_rng(31)
    d_old = oracle.sssp(g["offsets"], g["indices"], g["weights"], 0)
    gn, seeds = shorten(g, rng, 0.02, 300)
    d, st = run_warm(llp, gn, 0, d_old, seeds, **kw)
    assert (d == oracle.sssp(gn["offsets"], gn["indices"], gn["weights"], 0)).all()


@pytest.mark.parametrize("seed", range(6))
def test_warm_random_graphs(llp, seed):
    rng = np.random.default_rng(800 + seed)
    n = int(rng.integers(2, 4000))
    arcs = [(int(rng.integers(n)), int(rng.integers(n)), int(rng.integers(1, 1000)))
            for _ in range(int(rng.integers(0, 5 * n)))]
    arcs += [(0, int(rng.integers(n)), int(rng.integers(1, 50))) for _ in range(int(rng.integers(0, 800)))]
    g = csr_from_arcs(n, arcs)
    s = int(rng.integers(n))
    d_old = oracle.sssp(g["offsets"], g["indices"], g["weights"], s)
    gn, seeds = shorten(g, rng, float(rng.random()) * 0.2, int(rng.integers(0, n)), 1000)
    ref = oracle.sssp(gn["offsets"], gn["indices"], gn["weights"], s)
    d, _ = run_warm(llp, gn, s, d_old, seeds, offsets_64=bool(seed % 2))
    assert (d == ref).all()
    # BFS after the same insertions (levels only shrink)
    lv_old = oracle.bfs(g["offsets"], g["indices"], s)
    lv, _ = run_warm(llp, gn, s, lv_old, seeds, unit=True)
    assert (lv == oracle.bfs(gn["offsets"], gn["indices"], s)).all()


def test_warm_grid_and_rmat(llp):
    for g, s in ((synth.grid_graph(64, 80, 1, 1000, seed=3), 0), (synth.rmat(16, seed=21), None)):
        s = synth.max_out_degree_vertex(g) if s is None else s
        rng = np.random.default_rng(5)
        d_old = oracle.sssp(g["offsets"], g["indices"], g["weights"], s)
        gn, seeds = shorten(g, rng, 0.01, 50, 255)
        d, _ = run_warm(llp, gn, s, d_old, seeds)
        assert (d == oracle.sssp(gn["offsets"], gn["indices"], gn["weights"], s)).all()


def test_warm_without_changes_and_from_scratch_state(llp):
    g = synth.er16k()
    ref = oracle.sssp(g["offsets"], g["indices"], g["weights"], 0)
    d, st = run_warm(llp, g, 0, ref, None)  # nothing changed: the state is already the fixed point
    assert (d == ref).all() and st["advances"] == 0
    # the bottom state with the source as the only seed is the cold start
    bottom = np.full(g["n"], oracle.INF, np.uint32)
    d, _ = run_warm(llp, g, 0, bottom, np.array([0], np.int32))
    assert (d == ref).all()


def test_warm_invalid_seed_reported(llp):
    g = synth.er16k()
    ref = oracle.sssp(g["offsets"], g["indices"], g["weights"], 0)
    dg = dev_graph(llp, g)
    dist = torch.from_numpy(ref.view(np.int32).copy()).cuda()
    _, ws = llp.sssp_warm(dg, 0, dist, torch.tensor([3, g["n"]], dtype=torch.int32, device="cuda"))
    assert llp.get_status(ws)["status"] == llp.LLP_ERR_INVALID_ARG


# ------------------------------------------------------ host-buffer entry point

@pytest.mark.parametrize("pinned,off64", [(True, False), (False, False), (True, True)])
def test_sssp_host_buffers(llp, pinned, off64):
    for g, s in ((synth.er16k(), 0), (synth.rmat(16, seed=21), None)):
        s = synth.max_out_degree_vertex(g) if s is None else s
        off = torch.from_numpy(g["offsets"].astype(np.int64 if off64 else np.int32))
        idx = torch.from_numpy(g["indices"])
        w = torch.from_numpy(g["weights"].view(np.int32))
        out = torch.full((g["n"],), 7, dtype=torch.int32)
        if pinned:
            off, idx, w, out = off.pin_memory(), idx.pin_memory(), w.pin_memory(), out.pin_memory()
        _, ws = llp.sssp_host(off, idx, w, s, out)
        st = llp.get_status(ws)  # synchronises the stream
        assert st["status"] == 0
        assert (out.numpy().view(np.uint32) == oracle.sssp(g["offsets"], g["indices"], g["weights"], s)).all()


def test_sssp_host_rejects_device_tensors(llp):
    g = synth.er16k()
    off = torch.from_numpy(g["offsets"].astype(np.int32))
    with pytest.raises(ValueError):
        llp.sssp_host(off.cuda(), torch.from_numpy(g["indices"]), torch.from_numpy(g["weights"].view(np.int32)), 0,
                      torch.empty(g["n"], dtype=torch.int32))


def test_stats_report_the_schedule_used(llp):
    """llp_stats_t echoes the schedule the run used (mode, bucket width, block configuration,
    local chain) and counts its dense sweeps."""
    g = synth.er16k()
    ref = oracle.sssp(g["offsets"], g["indices"], g["weights"], 0)
    d, st = run_sssp(llp, g, 0, mode=1, delta=64, block_cfg=3, local_chain=16)
    assert (d == ref).all()
    assert (st["mode_used"], st["delta_used"], st["block_cfg_used"], st["local_chain_used"]) == (1, 64, 3, 16)
    assert st["dense_sweeps"] == 0 and st["pull_sweeps"] == 0
    d, st = run_sssp(llp, g, 0, mode=2)
    assert (d == ref).all()
    assert st["mode_used"] == 2 and st["local_chain_used"] == 0 and st["delta_used"] == llp.DELTA_INF
    assert st["dense_sweeps"] == st["sweeps"] - 2  # all but the first (list) and the last (empty) sweep


@pytest.mark.parametrize("m_extra", [0, 1, 3])
def test_gather_floor_reads_every_arc(llp, m_extra):
    """The access-pattern floor pass touches every arc once: the minimum over its per-thread
    results is min over arcs of state[target] + weight (vector body and the ragged tail)."""
    g = synth.er_graph(5000, 40000 + m_extra, 1, 100, seed=4)
    dg = dev_graph(llp, g)
    rng = np.random.default_rng(1)
    state = rng.integers(0, 1 << 20, g["n"]).astype(np.int32)
    sink = llp.gather_floor(dg, torch.from_numpy(state).cuda())
    got = int(sink.view(torch.int64).cpu().numpy().view(np.uint64).min())
    want = int((state[g["indices"]].astype(np.uint64) + g["weights"].astype(np.uint64)).min())
    assert got == want
    # one target made cheap at a time: the first arc, a middle one and the last (the tail)
    for e in (0, g["m"] // 2, g["m"] - 1):
        st2 = np.full(g["n"], 1 << 30, np.int32)
        v = g["indices"][e]
        st2[v] = 0
        sink = llp.gather_floor(dg, torch.from_numpy(st2).cuda(), sink=sink)
        got = int(sink.view(torch.int64).cpu().numpy().view(np.uint64).min())
        assert got == int(g["weights"][g["indices"] == v].min()), e
