"""GPU parity (through the C ABI) of stable marriage, knapsack, job scheduling,
transitive closure and reduction against the oracle, bit-exact."""
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


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# ---------------------------------------------------------- stable marriage

def check_marriage(llp, mp, wr):
    wife, hus, nxt, ws = llp.stable_marriage(T(mp), T(wr))
    st = llp.get_status(ws)
    assert st["status"] == 0, st
    rw, rh, rn, props = oracle.stable_marriage(mp, wr)
    assert (wife.cpu().numpy() == rw).all()
    assert (hus.cpu().numpy() == rh).all()
    assert (nxt.cpu().numpy() == rn).all()  # the LLP state G is unique too
    return st, props


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (7, 2), (100, 3), (1000, 4), (1023, 5)])
def test_marriage_random(llp, n, seed):
    mp, wr = synth.marriage(n, seed=seed)
    check_marriage(llp, mp, wr)


def test_marriage_shared_order(llp):
    mp, wr = synth.marriage(1500, seed=9, adversarial=True)
    st, props = check_marriage(llp, mp, wr)
    assert props == 1500 * 1501 // 2


def test_marriage_malformed_is_infeasible(llp):
    # a list that repeats a woman: the man runs off the end of his list
    mp = np.array([[0, 0], [0, 0]], np.int32)
    wr = np.array([[0, 1], [0, 1]], np.int32)
    _, _, _, ws = llp.stable_marriage(T(mp), T(wr))
    assert llp.get_status(ws)["status"] == llp.LLP_ERR_INFEASIBLE


@pytest.mark.slow
def test_marriage_full_random_16384(llp):
    mp, wr = synth.marriage(16384, seed=3)
    check_marriage(llp, mp, wr)


@pytest.mark.slow
def test_marriage_full_adversarial_8192(llp):
    mp, wr = synth.marriage(8192, seed=4, adversarial=True)
    st, props = check_marriage(llp, mp, wr)
    assert props == 8192 * 8193 // 2 == st["aux"]


# ------------------------------------------------------------------ knapsack

@pytest.mark.parametrize("n,W,seed", [(0, 10, 0), (1, 0, 1), (5, 3, 2), (40, 1000, 3), (300, 4096, 4),
                                      (2048, 65536, 5), (17, 60000, 6), (500, 57343, 7)])
def test_knapsack(llp, n, W, seed):
    w, v = synth.knapsack(n, W, seed=seed) if n else (np.zeros(0, np.int32), np.zeros(0, np.int32))
    if n and seed == 2:
        w[:] = 5  # nothing fits
    best, row, ws = llp.knapsack(T(w) if n else torch.zeros(0, dtype=torch.int32, device="cuda"),
                                 T(v) if n else torch.zeros(0, dtype=torch.int32, device="cuda"), W)
    assert llp.get_status(ws)["status"] == 0
    rb, rrow = oracle.knapsack(w, v, W)
    assert int(best.item()) == rb
    assert (row.cpu().numpy() == rrow).all()


@pytest.mark.parametrize("n,W,seed,cfg", [(2048, 65536, 5, 1), (1000, 30000, 8, 0), (1001, 65536, 9, 0),
                                          (2000, 200000, 10, 0), (4096, 4096, 11, 0), (3, 100000, 12, 0),
                                          (2048, 65536, 5, 3), (1001, 65536, 9, 3), (2000, 200000, 10, 3),
                                          (8000, 65536, 14, 0), (4099, 5000, 15, 0), (1500, 1000000, 16, 0)])
def test_knapsack_wavefront_cluster_and_single_cta(llp, n, W, seed, cfg):
    """Large instances run as a wavefront over capacity slices (one CTA per slice, rows exchanged
    through a tagged ring in global memory: ragged item counts leave a partial last block, more
    items than ring rows wrap it, a large capacity takes several cells per thread); block_cfg 3
    runs the thread-block cluster kernel (rows in distributed shared memory, two items per pass)
    and block_cfg 1 the one-CTA kernel on the same instance."""
    w, v = synth.knapsack(n, W, seed=seed)
    best, row, ws = llp.knapsack(T(w), T(v), W, sched=llp.make_sched(block_cfg=cfg))
    assert llp.get_status(ws)["status"] == 0
    rb, rrow = oracle.knapsack(w, v, W)
    assert int(best.item()) == rb
    assert (row.cpu().numpy() == rrow).all()


def test_knapsack_wave_invalid_item_reported(llp):
    """An item outside the problem statement (weight 0) is skipped and reported on the wavefront path."""
    w, v = synth.knapsack(2048, 65536, seed=13)
    w[100] = 0
    best, row, ws = llp.knapsack(T(w), T(v), 65536)
    assert llp.get_status(ws)["status"] == llp.LLP_ERR_INVALID_ARG
    keep = np.ones(2048, bool)
    keep[100] = False
    assert int(best.item()) == oracle.knapsack(w[keep], v[keep], 65536)[0]


def test_knapsack_overflow_reported(llp):
    w = np.ones(4, np.int32)
    v = np.full(4, 0x7FFFFFFF // 3, np.int32)
    _, _, ws = llp.knapsack(T(w), T(v), 10)
    assert llp.get_status(ws)["status"] == llp.LLP_ERR_OVERFLOW


# ------------------------------------------------------------- job schedule

def job_dev(llp, g):
    return llp.DeviceGraph.from_host(g, "cuda")


def test_job_paper_example(llp):
    gd = read_golden("job_race_example.txt")
    dur = np.array([int(x) for x in gd["duration"][0].split()], np.int32)
    g = dict(n=3, m=2, offsets=np.array([0, 1, 2, 2], np.int64), indices=np.array([2, 2], np.int32), weights=None)
    c, ws = llp.job_schedule(job_dev(llp, g), T(dur))
    assert llp.get_status(ws)["status"] == 0
    assert c.cpu().numpy().tolist() == [int(x) for x in gd["completion"][0].split()]


@pytest.mark.parametrize("n,seed", [(1, 0), (64, 1), (5000, 2), (8192, 3), (200000, 4), (1 << 20, 5)])
def test_job_random(llp, n, seed):
    """Random job DAGs up to the benchmarked 1,048,576-job DAG (the same seed)."""
    g, dur = synth.job_dag(n, seed=seed)
    c, ws = llp.job_schedule(job_dev(llp, g), T(dur))
    st = llp.get_status(ws)
    assert st["status"] == 0, st
    assert (c.cpu().numpy() == oracle.job_schedule(dur, g["offsets"], g["indices"])).all()


def test_job_int64_offsets(llp):
    g, dur = synth.job_dag(20000, seed=9)
    c, ws = llp.job_schedule(llp.DeviceGraph.from_host(g, "cuda", offsets_64=True), T(dur))
    assert llp.get_status(ws)["status"] == 0
    assert (c.cpu().numpy() == oracle.job_schedule(dur, g["offsets"], g["indices"])).all()


@pytest.mark.parametrize("fan", [5000, 100000])
def test_job_wide_ready_sets(llp, fan):
    """A job with `fan` successors, each with one more successor: one warp makes all of them
    ready in one sweep, more than a CTA stages in shared memory (the rest spill to the list)."""
    rng = np.random.default_rng(fan)
    n = 1 + 2 * fan
    src = np.concatenate([np.zeros(fan, np.int64), np.arange(1, fan + 1)])
    dst = np.concatenate([np.arange(1, fan + 1), np.arange(fan + 1, n)])
    offsets = np.zeros(n + 1, np.int64)
    np.add.at(offsets, src + 1, 1)
    offsets = np.cumsum(offsets)
    indices = dst[np.argsort(src, kind="stable")].astype(np.int32)
    g = dict(n=n, m=len(indices), offsets=offsets, indices=indices, weights=None)
    dur = rng.integers(1, 101, n).astype(np.int32)
    c, ws = llp.job_schedule(job_dev(llp, g), T(dur))
    st = llp.get_status(ws)
    assert st["status"] == 0, st
    assert (c.cpu().numpy() == oracle.job_schedule(dur, offsets, indices)).all()


def test_job_cycle_is_infeasible(llp):
    g = dict(n=3, m=3, offsets=np.array([0, 1, 2, 3], np.int64), indices=np.array([1, 2, 0], np.int32), weights=None)
    _, ws = llp.job_schedule(job_dev(llp, g), T(np.ones(3, np.int32)))
    assert llp.get_status(ws)["status"] == llp.LLP_ERR_INFEASIBLE


# ------------------------------------------------------- transitive closure

@pytest.mark.parametrize("n,seed", [(1, 0), (5, 1), (33, 2), (500, 3)])
def test_closure_random_with_cycles(llp, n, seed):
    rng = np.random.default_rng(seed)
    m = int(rng.integers(0, 3 * n + 1))
    src = rng.integers(0, n, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)
    order = np.argsort(src, kind="stable")
    off = np.zeros(n + 1, np.int64)
    np.add.at(off, src + 1, 1)
    g = dict(n=n, m=m, offsets=np.cumsum(off), indices=dst[order], weights=None)
    R, ws = llp.transitive_closure(llp.DeviceGraph.from_host(g, "cuda"))
    assert llp.get_status(ws)["status"] == 0
    assert (R.cpu().numpy().view(np.uint32) == oracle.transitive_closure(g["offsets"], g["indices"])).all()


def test_closure_int64_offsets_and_chain(llp):
    n = 300
    g = dict(n=n, m=n - 1, offsets=np.concatenate([np.arange(n, dtype=np.int64), [n - 1]]),
             indices=np.arange(1, n, dtype=np.int32), weights=None)
    R, ws = llp.transitive_closure(llp.DeviceGraph.from_host(g, "cuda", offsets_64=True))
    assert llp.get_status(ws)["status"] == 0
    bits = np.unpackbits(R.cpu().numpy().view(np.uint8), axis=1, bitorder="little")[:, :n].astype(bool)
    assert (bits == np.triu(np.ones((n, n), bool), 1)).all()  # closure of a chain


def test_closure_random_dag_8192(llp):
    """Closure workload: random DAG n=8192, arc probability 4/n."""
    g = synth.random_dag(8192, 4, seed=6)
    R, ws = llp.transitive_closure(llp.DeviceGraph.from_host(g, "cuda"))
    st = llp.get_status(ws)
    assert st["status"] == 0
    ref = oracle.transitive_closure(g["offsets"], g["indices"])
    assert (R.cpu().numpy().view(np.uint32) == ref).all()


# ---------------------------------------------------------------- reduction

@pytest.mark.parametrize("n", [0, 1, 3, 1000, 8191, 8193, (1 << 24) + 5, 100_000_007])
def test_reduce(llp, n):
    x = synth.u64(n, seed=n % 97)
    out, ws = llp.reduce_sum(T(x.view(np.int64)))
    assert llp.get_status(ws)["status"] == 0
    assert int(out.cpu().numpy().view(np.uint64)[0]) == oracle.reduce_sum(x)


def test_reduce_closed_form(llp):
    n = (1 << 22) + 3
    x = np.arange(n, dtype=np.uint64)
    out, _ = llp.reduce_sum(T(x.view(np.int64)))
    assert int(out.cpu().numpy().view(np.uint64)[0]) == n * (n - 1) // 2
