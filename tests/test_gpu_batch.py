"""GPU parity of the batched engine (one persistent launch over many instances)
against the oracle, bit-exact, including CUDA-graph capture and the autotuner."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def llp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_13147_b300 as m
    m.lib()
    return m


def small_batches(seed=0, kc=40, jc=30, sc=30):
    knap = synth.knapsack_batch(kc, 0, 200, 0, 3000, seed=seed) if kc else None
    if knap is not None:
        # two instances above the shared-memory row size (global-memory row path)
        knap["capacity"][:2] = [60000, 65536]
    job = synth.job_batch(jc, 1, 3000, seed=seed) if jc else None
    sm = synth.marriage_batch(sc, 1, 300, seed=seed) if sc else None
    return knap, job, sm


def check_knap(db, knap, idx):
    best = db.t["knap_best"].cpu().numpy()
    for i in idx:
        a, b = knap["item_off"][i], knap["item_off"][i + 1]
        assert best[i] == oracle.knapsack(knap["w"][a:b], knap["v"][a:b], int(knap["capacity"][i]))[0], i


def check_job(db, job, idx):
    comp = db.t["job_completion"].cpu().numpy()
    for i in idx:
        j0, j1 = job["job_off"][i], job["job_off"][i + 1]
        off = job["succ_offsets"][j0:j1 + 1] - job["succ_offsets"][j0]
        ind = job["succ_indices"][job["succ_offsets"][j0]:job["succ_offsets"][j1]]
        assert (comp[j0:j1] == oracle.job_schedule(job["duration"][j0:j1], off, ind)).all(), i


def check_sm(db, sm, idx):
    wife = db.t["sm_wife"].cpu().numpy()
    mo = db.sm_man_off_host
    for i in idx:
        n = int(sm["n"][i])
        p0 = sm["pref_off"][i]
        mp = sm["men_pref"][p0:p0 + n * n].reshape(n, n)
        wr = sm["women_rank"][p0:p0 + n * n].reshape(n, n)
        assert (wife[mo[i]:mo[i + 1]] == oracle.stable_marriage(mp, wr)[0]).all(), i


@pytest.mark.parametrize("threads,unroll,ctas", [(1024, 8, 1), (512, 4, 1), (256, 16, 1), (512, 8, 2), (256, 4, 2)])
def test_batch_small_all_instances(llp, threads, unroll, ctas):
    knap, job, sm = small_batches(seed=threads + ctas)
    db = llp.DeviceBatch(knap, job, sm)
    cfg = llp.BatchCfg()
    cfg.threads, cfg.knap_unroll, cfg.ctas_per_sm = threads, unroll, ctas
    ws = llp.batch_solve(db, cfg)
    st = llp.get_status(ws)
    assert st["status"] == 0, st
    assert st["items"] == db.count
    check_knap(db, knap, range(knap["count"]))
    check_job(db, job, range(job["count"]))
    check_sm(db, sm, range(sm["count"]))


def test_batch_single_family_and_empty(llp):
    knap, _, _ = small_batches(seed=3, jc=0, sc=0)
    db = llp.DeviceBatch(knap, None, None)
    ws = llp.batch_solve(db)
    assert llp.get_status(ws)["status"] == 0
    check_knap(db, knap, range(knap["count"]))
    empty = llp.DeviceBatch(None, None, None)
    llp.batch_solve(empty)


def test_batch_cuda_graph_replay(llp):
    knap, job, sm = small_batches(seed=5, kc=20, jc=20, sc=20)
    db = llp.DeviceBatch(knap, job, sm)
    ws = llp.workspace(llp.batch_workspace_size(db))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        llp.batch_solve(db, ws=ws, stream=s)  # warm (loads the kernels)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        llp.batch_solve(db, ws=ws, stream=s)
    for t in ("knap_best", "job_completion", "sm_wife"):
        db.t[t].fill_(-7)
    g.replay()
    torch.cuda.synchronize()
    assert llp.get_status(ws)["status"] == 0
    check_knap(db, knap, range(knap["count"]))
    check_job(db, job, range(job["count"]))
    check_sm(db, sm, range(sm["count"]))


def test_batch_autotune_picks_a_candidate(llp):
    knap, job, sm = small_batches(seed=9, kc=30, jc=10, sc=10)
    db = llp.DeviceBatch(knap, job, sm)
    best, ms, ws = llp.batch_autotune(db)
    assert len(ms) == 12 and best.threads in (256, 512, 1024) and best.knap_unroll in (4, 8, 16)
    assert best.ctas_per_sm in (1, 2)
    assert min(ms) > 0
    check_knap(db, knap, range(knap["count"]))


@pytest.mark.slow
def test_batch_full_config_sampled(llp):
    """Full batched workload: 4,096 knapsack + 2,048 job DAGs + 1,024 marriages, one launch;
    parity on a seeded sample of instances of each family."""
    knap = synth.knapsack_batch()
    job = synth.job_batch()
    sm = synth.marriage_batch()
    db = llp.DeviceBatch(knap, job, sm)
    ws = llp.batch_solve(db)
    st = llp.get_status(ws)
    assert st["status"] == 0, st
    assert st["items"] == 4096 + 2048 + 1024
    rng = np.random.default_rng(0)
    cells = np.diff(knap["item_off"]) * (knap["capacity"].astype(np.int64) + 1)
    largest = np.argsort(cells)[-4:]  # the biggest n * W instances, then a seeded sample
    check_knap(db, knap, np.unique(np.concatenate([largest, rng.choice(4096, 60, replace=False)])))
    jobs = np.diff(job["job_off"])
    check_job(db, job, np.unique(np.concatenate([np.argsort(jobs)[-4:], rng.choice(2048, 64, replace=False)])))
    check_sm(db, sm, np.unique(np.concatenate([np.argsort(sm["n"])[-4:], rng.choice(1024, 48, replace=False)])))


# ----------------------------------------------------- small SSSP / BFS family

def check_graphs(db, gb, idx):
    dist = db.t["gr_dist"].cpu().numpy().view(np.uint32)
    for i in idx:
        v0, v1 = gb["off"][i], gb["off"][i + 1]
        off = gb["arc_offsets"][v0:v1 + 1] - gb["arc_offsets"][v0]
        a, b = gb["arc_offsets"][v0], gb["arc_offsets"][v1]
        idx_ = gb["indices"][a:b]
        s = int(gb["source"][i])
        if gb["unit"] is not None and gb["unit"][i]:
            ref = oracle.bfs(off, idx_, s)
        else:
            ref = oracle.sssp(off, idx_, gb["weights"][a:b], s)
        assert (dist[v0:v1] == ref).all(), i


@pytest.mark.parametrize("threads,unroll,ctas", [(1024, 8, 1), (512, 4, 1), (256, 16, 1), (512, 16, 2)])
def test_batch_graphs_with_other_families(llp, threads, unroll, ctas):
    knap, job, sm = small_batches(seed=threads + 1, kc=10, jc=10, sc=10)
    gb = synth.graph_batch(48, 1, 4000, seed=threads)
    db = llp.DeviceBatch(knap, job, sm, gb)
    cfg = llp.BatchCfg()
    cfg.threads, cfg.knap_unroll, cfg.ctas_per_sm = threads, unroll, ctas
    ws = llp.batch_solve(db, cfg)
    st = llp.get_status(ws)
    assert st["status"] == 0, st
    assert st["items"] == db.count
    check_graphs(db, gb, range(gb["count"]))
    check_knap(db, knap, range(knap["count"]))
    check_job(db, job, range(job["count"]))
    check_sm(db, sm, range(sm["count"]))


def test_batch_graphs_above_shared_memory(llp):
    """Instances whose d[] and bitmaps exceed shared memory work on the output in place."""
    gb = synth.graph_batch(8, 56000, 90000, seed=17)
    db = llp.DeviceBatch(graphs=gb)
    ws = llp.batch_solve(db)
    assert llp.get_status(ws)["status"] == 0
    check_graphs(db, gb, range(gb["count"]))


def test_batch_graph_edge_cases(llp):
    # one vertex without arcs; a source without out-arcs; self-loops and parallel arcs; BFS and SSSP
    insts = [(1, [], 0, 0), (5, [(1, 2, 3), (2, 3, 4)], 0, 0),
             (3, [(0, 0, 1), (0, 1, 9), (0, 1, 4), (1, 1, 2), (1, 2, 7), (1, 2, 5)], 0, 0),
             (3, [(0, 0, 1), (0, 1, 9), (0, 1, 4), (1, 1, 2), (1, 2, 7), (1, 2, 5)], 0, 1),
             (4, [(3, 2, 1), (2, 1, 1), (1, 0, 1)], 3, 0)]
    verts, arc_off, idxs, ws_, srcs, unit = [0], [], [], [], [], []
    base = 0
    for n, arcs, s, u in insts:
        arcs = sorted(arcs, key=lambda t: t[0])
        off = np.zeros(n + 1, np.int64)
        for a in arcs:
            off[a[0] + 1] += 1
        off = np.cumsum(off)
        arc_off.append(off[:-1] + base)
        idxs += [a[1] for a in arcs]
        ws_ += [a[2] for a in arcs]
        base += len(arcs)
        verts.append(verts[-1] + n)
        srcs.append(s)
        unit.append(u)
    gb = dict(count=len(insts), off=np.array(verts, np.int64),
              arc_offsets=np.concatenate(arc_off + [np.array([base], np.int64)]),
              indices=np.array(idxs, np.int32), weights=np.array(ws_, np.uint32), source=np.array(srcs, np.int32),
              unit=np.array(unit, np.int32))
    db = llp.DeviceBatch(graphs=gb)
    ws = llp.batch_solve(db)
    assert llp.get_status(ws)["status"] == 0
    d = db.t["gr_dist"].cpu().numpy().view(np.uint32).tolist()
    INF = oracle.INF
    assert d == [0] + [0, INF, INF, INF, INF] + [0, 4, 9] + [0, 1, 2] + [3, 2, 1, 0]


def test_batch_graph_overflow_and_bad_source(llp):
    def one(n, arcs, s):
        off = np.zeros(n + 1, np.int64)
        for a in arcs:
            off[a[0] + 1] += 1
        return dict(count=1, off=np.array([0, n], np.int64), arc_offsets=np.cumsum(off),
                    indices=np.array([a[1] for a in arcs], np.int32),
                    weights=np.array([a[2] for a in arcs], np.uint32), source=np.array([s], np.int32), unit=None)
    db = llp.DeviceBatch(graphs=one(3, [(0, 1, 0xF0000000), (1, 2, 0xF0000000)], 0))
    assert llp.get_status(llp.batch_solve(db))["status"] == llp.LLP_ERR_OVERFLOW
    db = llp.DeviceBatch(graphs=one(3, [(0, 1, 1)], 3))
    assert llp.get_status(llp.batch_solve(db))["status"] == llp.LLP_ERR_INVALID_ARG


def test_batch_graphs_cuda_graph_replay(llp):
    gb = synth.graph_batch(32, 1, 3000, seed=23)
    db = llp.DeviceBatch(graphs=gb)
    ws = llp.workspace(llp.batch_workspace_size(db))
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        llp.batch_solve(db, ws=ws, stream=s)
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        llp.batch_solve(db, ws=ws, stream=s)
    db.t["gr_dist"].fill_(-7)
    g.replay()
    torch.cuda.synchronize()
    assert llp.get_status(ws)["status"] == 0
    check_graphs(db, gb, range(gb["count"]))


@pytest.mark.slow
def test_batch_graphs_2048_sampled(llp):
    """The batched small-graph workload of the benchmark: 2,048 graphs of 64-8,192 vertices."""
    gb = synth.graph_batch()
    db = llp.DeviceBatch(graphs=gb)
    ws = llp.batch_solve(db)
    st = llp.get_status(ws)
    assert st["status"] == 0 and st["items"] == 2048
    rng = np.random.default_rng(1)
    check_graphs(db, gb, rng.choice(2048, 96, replace=False))
