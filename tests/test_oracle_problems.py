"""Pins of the stable-marriage, knapsack, job-scheduling, reduction and MLP oracles."""
import itertools

import numpy as np
import pytest

import oracle
import oracle.mlp as omlp
import synth
from conftest import read_golden


# ---------------------------------------------------------- stable marriage

def blocking_pairs(men_pref, women_rank, wife):
    n = len(wife)
    husband = np.empty(n, int)
    husband[wife] = np.arange(n)
    mrank = np.empty((n, n), int)
    for m in range(n):
        mrank[m, men_pref[m]] = np.arange(n)
    out = []
    for m in range(n):
        for w in range(n):
            if mrank[m, w] < mrank[m, wife[m]] and women_rank[w, m] < women_rank[w, husband[w]]:
                out.append((m, w))
    return out


def stable_matchings_brute(men_pref, women_rank):
    n = men_pref.shape[0]
    return [np.array(p) for p in itertools.permutations(range(n))
            if not blocking_pairs(men_pref, women_rank, np.array(p))]


@pytest.mark.parametrize("seed", range(25))
def test_marriage_man_optimal_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 8))
    mp = np.stack([rng.permutation(n) for _ in range(n)]).astype(np.int32)
    wr = np.stack([np.argsort(rng.permutation(n)) for _ in range(n)]).astype(np.int32)
    wife, hus, nxt, _ = oracle.stable_marriage(mp, wr)
    stable = stable_matchings_brute(mp, wr)
    assert any((s == wife).all() for s in stable)
    # man-optimal: every man's partner is his best over all stable matchings
    mrank = np.argsort(mp, axis=1)
    for m in range(n):
        assert mrank[m, wife[m]] == min(mrank[m, s[m]] for s in stable)
    assert (hus[wife] == np.arange(n)).all()
    assert (mp[np.arange(n), nxt] == wife).all()


def test_marriage_no_blocking_pair_random():
    mp, wr = synth.marriage(150, seed=11)
    wife, _, _, _ = oracle.stable_marriage(mp, wr)
    assert sorted(wife.tolist()) == list(range(150))
    assert blocking_pairs(mp, wr, wife) == []


def test_marriage_shared_order_closed_form():
    """All men share one order w0, w1, ...: woman w_k ends with her favourite man
    among those not taken by w_0..w_{k-1}, and there are n(n+1)/2 proposals."""
    n = 60
    mp, wr = synth.marriage(n, seed=4, adversarial=True)
    order = mp[0]
    assert (mp == order).all()
    wife, _, _, props = oracle.stable_marriage(mp, wr)
    assert props == n * (n + 1) // 2
    free = set(range(n))
    for w in order:
        fav = min(free, key=lambda m: wr[w, m])
        assert wife[fav] == w
        free.remove(fav)


# ------------------------------------------------------------------ knapsack

def knap_brute(w, v, W):
    n = len(w)
    best = [0] * (W + 1)
    for mask in range(1 << n):
        tw = sum(w[i] for i in range(n) if mask >> i & 1)
        tv = sum(v[i] for i in range(n) if mask >> i & 1)
        for c in range(tw, W + 1):
            if tv > best[c]:
                best[c] = tv
    return best


@pytest.mark.parametrize("seed", range(25))
def test_knapsack_brute_force(seed):
    rng = np.random.default_rng(400 + seed)
    n = int(rng.integers(0, 13))
    W = int(rng.integers(0, 60))
    w = rng.integers(1, 25, n).astype(np.int32)
    v = rng.integers(1, 1000, n).astype(np.int32)
    best, row = oracle.knapsack(w, v, W)
    bf = knap_brute(w.tolist(), v.tolist(), W)
    assert best == bf[W]
    assert row.tolist() == bf


def test_knapsack_brute_force_n20():
    rng = np.random.default_rng(7)
    w = rng.integers(1, 40, 20).astype(np.int32)
    v = rng.integers(1, 1000, 20).astype(np.int32)
    W = 150
    tw = np.array([[mask >> i & 1 for i in range(20)] for mask in range(1 << 20)], np.int64)
    ws, vs = tw @ w, tw @ v
    assert oracle.knapsack(w, v, W)[0] == int(vs[ws <= W].max())


def test_knapsack_special_cases():
    rng = np.random.default_rng(8)
    v = rng.integers(1, 1000, 300).astype(np.int32)
    for W in (0, 1, 17, 299, 300, 1000):
        best, _ = oracle.knapsack(np.ones(300, np.int32), v, W)
        assert best == int(np.sort(v)[::-1][:min(300, W)].sum())
    w = rng.integers(1, 100, 300).astype(np.int32)
    W = 2000
    best, _ = oracle.knapsack(w, np.full(300, 7, np.int32), W)
    cnt = int((np.cumsum(np.sort(w)) <= W).sum())
    assert best == 7 * cnt


# ------------------------------------------------------------- job schedule

def job_brute(n, dur, arcs):
    """Max over all paths ending at j of the sum of durations on the path."""
    preds = [[] for _ in range(n)]
    for u, v in arcs:
        preds[v].append(u)

    def best(j):
        return dur[j] + max([best(p) for p in preds[j]], default=0)

    return [best(j) for j in range(n)]


def csr(n, arcs):
    arcs = sorted(enumerate(arcs), key=lambda t: (t[1][0], t[0]))
    off = np.zeros(n + 1, np.int64)
    for _, a in arcs:
        off[a[0] + 1] += 1
    return np.cumsum(off), np.array([a[1] for _, a in arcs], np.int32)


def test_job_paper_race_example():
    g = read_golden("job_race_example.txt")
    dur = np.array([int(x) for x in g["duration"][0].split()], np.int32)
    arcs = [tuple(int(x) for x in a.split()) for a in g["arc"]]
    off, idx = csr(3, arcs)
    assert oracle.job_schedule(dur, off, idx).tolist() == [int(x) for x in g["completion"][0].split()]


@pytest.mark.parametrize("seed", range(25))
def test_job_brute_force(seed):
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(1, 9))
    perm = rng.permutation(n)  # random topological labelling
    arcs = [(int(perm[i]), int(perm[j])) for i in range(n) for j in range(i + 1, n) if rng.random() < 0.4]
    dur = rng.integers(0, 50, n).astype(np.int32)
    off, idx = csr(n, arcs)
    assert oracle.job_schedule(dur, off, idx).tolist() == job_brute(n, dur.tolist(), arcs)


def test_job_invariants_and_cycle():
    g, dur = synth.job_dag(3000, seed=12)
    c = oracle.job_schedule(dur, g["offsets"], g["indices"])
    src = np.repeat(np.arange(g.n), np.diff(g["offsets"]))
    assert (c[g["indices"]] >= c[src] + dur[g["indices"]]).all()
    # tight: c[j] == dur[j] or some predecessor p has c[p] + dur[j] == c[j]
    tight = c == dur
    ok = c[src] + dur[g["indices"]] == c[g["indices"]]
    tight[g["indices"][ok]] = True
    assert tight.all()
    off, idx = csr(3, [(0, 1), (1, 2), (2, 0)])
    with pytest.raises(oracle.OracleError) as e:
        oracle.job_schedule(np.ones(3, np.int32), off, idx)
    assert e.value.code == oracle.ERR_CYCLE


# ------------------------------------------------------------------ reduce

def test_reduce_closed_form_and_wrap():
    n = 1 << 20
    assert oracle.reduce_sum(np.arange(n, dtype=np.uint64)) == n * (n - 1) // 2
    assert oracle.reduce_sum(np.array([2 ** 64 - 1, 2], np.uint64)) == 1
    x = synth.u64(10000, seed=3)
    assert oracle.reduce_sum(x) == sum(int(a) for a in x) % (1 << 64)
    assert oracle.reduce_sum(np.zeros(0, np.uint64)) == 0


# --------------------------------------------------------------------- MLP

def test_mlp_gradient_finite_differences():
    F, H1, H2, O = 5, 7, 6, 9
    heads = [2, 4, 3]
    rng = np.random.default_rng(1)
    nparam = F * H1 + H1 + H1 * H2 + H2 + H2 * O + O
    th = rng.normal(0, 0.5, nparam)
    X = rng.normal(0, 1, (11, F))
    Y = np.stack([rng.integers(0, h, 11) for h in heads], axis=1)
    L, g = omlp.backward(th, X, Y, heads, F, H1, H2, O)
    assert abs(L - omlp.loss(th, X, Y, heads, F, H1, H2, O)) < 1e-12
    eps = 1e-6
    for k in rng.choice(nparam, 60, replace=False):
        e = np.zeros(nparam); e[k] = eps
        fd = (omlp.loss(th + e, X, Y, heads, F, H1, H2, O) - omlp.loss(th - e, X, Y, heads, F, H1, H2, O)) / (2 * eps)
        assert abs(fd - g[k]) < 1e-6 * max(1.0, abs(fd))


def test_mlp_loss_closed_form_zero_weights():
    """All parameters zero: every head is uniform, loss = sum(log h)."""
    F, H1, H2, O = 4, 8, 8, 6
    heads = [2, 4]
    th = np.zeros(F * H1 + H1 + H1 * H2 + H2 + H2 * O + O)
    X = np.ones((3, F)); Y = np.zeros((3, 2), int)
    assert abs(omlp.loss(th, X, Y, heads, F, H1, H2, O) - (np.log(2) + np.log(4))) < 1e-12


def test_adam_first_step_closed_form():
    """First bias-corrected Adam step moves each parameter by lr*g/(|g|+eps)."""
    g = np.array([0.3, -2.0, 1e-3])
    th, m, v = omlp.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    assert np.allclose(th, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)


def test_mlp_forward_hand_worked():
    """Forward pass of a 2 -> 2 -> 2 -> 4 network worked out by hand.

    Layer 1 of sample 0: a1 = [1*1 + 2*0.5 + 0.5, 1*(-1) + 2*1 - 3] = [2.5, -2],
    the ReLU clips the second unit; layer 2: a2 = [2.5*1 - 3, 2.5*2 + 1] = [-0.5, 6],
    clipped again; logits = [6*0.5 + 1, 6*(-1), 6*0 - 2, 6*1 + 0.5].  A dropped
    bias, a missing ReLU on either layer or a transposed weight matrix changes them.
    """
    F, H1, H2, O = 2, 2, 2, 4
    W1 = [[1.0, -1.0], [0.5, 1.0]]          # W1[f, h]
    b1 = [0.5, -3.0]
    W2 = [[1.0, 2.0], [3.0, -1.0]]          # W2[h1, h2]
    b2 = [-3.0, 1.0]
    W3 = [[1.0, 0.0, 2.0, -1.0], [0.5, -1.0, 0.0, 1.0]]
    b3 = [1.0, 0.0, -2.0, 0.5]
    th = np.concatenate([np.ravel(a) for a in (W1, b1, W2, b2, W3, b3)])
    X = np.array([[1.0, 2.0], [0.0, -1.0]])
    z, _ = omlp.forward(th, X, F, H1, H2, O)
    # sample 1: a1 = [-0.5 + 0.5, -1 - 3] = [0, -4] -> h1 = 0, h2 = relu(b2) = [0, 1]
    assert np.array_equal(z, np.array([[4.0, -6.0, -2.0, 6.5], [1.5, -1.0, -2.0, 1.5]]))
    # two heads of 2 logits; labels (0, 1) and (1, 0): cross-entropy log(1 + e^(other - own))
    Y = np.array([[0, 1], [1, 0]])
    want = (np.log1p(np.exp(-10.0)) + np.log1p(np.exp(-8.5)) + np.log1p(np.exp(2.5)) + np.log1p(np.exp(3.5))) / 2
    assert abs(omlp.loss(th, X, Y, [2, 2], F, H1, H2, O) - want) < 1e-12
    assert np.array_equal(omlp.predict(th, X, [2, 2], F, H1, H2, O), np.array([[0, 1], [0, 1]]))


def test_adam_three_steps_hand_worked():
    """Three Adam steps (Kingma and Ba, Algorithm 1) on one parameter with gradients
    1, -2, 0.5, lr 0.1, beta1 0.9, beta2 0.999, worked by hand.  The bias
    corrections 1 - beta^t at t = 2, 3 are written out (0.19, 0.001999, 0.271,
    0.002997001), so a correction of the form 1 - beta*t cannot pass."""
    lr, eps = 0.1, 1e-8
    th, m, v = omlp.adam_step(np.zeros(1), np.array([1.0]), np.zeros(1), np.zeros(1), 1, lr=lr)
    assert abs(m[0] - 0.1) < 1e-15 and abs(v[0] - 0.001) < 1e-15
    th1 = -lr * 1.0 / (1.0 + eps)
    assert abs(th[0] - th1) < 1e-15
    th, m, v = omlp.adam_step(th, np.array([-2.0]), m, v, 2, lr=lr)
    # m2 = 0.9*0.1 + 0.1*(-2) = -0.11; v2 = 0.999*0.001 + 0.001*4 = 0.004999
    assert abs(m[0] + 0.11) < 1e-15 and abs(v[0] - 0.004999) < 1e-15
    th2 = th1 - lr * (-0.11 / 0.19) / (np.sqrt(0.004999 / 0.001999) + eps)
    assert abs(th[0] - th2) < 1e-13
    th, m, v = omlp.adam_step(th, np.array([0.5]), m, v, 3, lr=lr)
    # m3 = 0.9*(-0.11) + 0.1*0.5 = -0.049; v3 = 0.999*0.004999 + 0.001*0.25 = 0.005244001
    assert abs(m[0] + 0.049) < 1e-15 and abs(v[0] - 0.005244001) < 1e-15
    th3 = th2 - lr * (-0.049 / 0.271) / (np.sqrt(0.005244001 / 0.002997001) + eps)
    assert abs(th[0] - th3) < 1e-13
    assert abs(th[0] - (-0.0497206)) < 1e-6
