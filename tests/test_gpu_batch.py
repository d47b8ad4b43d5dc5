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


@pytest.mark.parametrize("threads,unroll", [(1024, 8), (512, 4), (256, 16)])
def test_batch_small_all_instances(llp, threads, unroll):
    knap, job, sm = small_batches(seed=threads)
    db = llp.DeviceBatch(knap, job, sm)
    cfg = llp.BatchCfg()
    cfg.threads, cfg.knap_unroll = threads, unroll
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
    assert len(ms) == 6 and best.threads in (512, 1024) and best.knap_unroll in (4, 8, 16)
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
    check_knap(db, knap, rng.choice(4096, 12, replace=False))
    check_job(db, job, rng.choice(2048, 64, replace=False))
    check_sm(db, sm, rng.choice(1024, 48, replace=False))
