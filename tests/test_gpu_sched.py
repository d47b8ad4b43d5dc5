"""Learned scheduler: GPU fp32 forward/backward/Adam against the fp64 CPU oracle,
on-device inference against the oracle network, and bit-exact results under any
schedule the network can choose."""
import os

import numpy as np
import pytest

import oracle
import oracle.mlp as omlp
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

F, H1, H2 = 16, 64, 64
HEADS = [3, 8, 3, 4, 5]
O = sum(HEADS)


@pytest.fixture(scope="module")
def llp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_13147_b300 as m
    m.lib()
    return m


def rand_problem(seed, B=37):
    rng = np.random.default_rng(seed)
    nparam = F * H1 + H1 + H1 * H2 + H2 + H2 * O + O
    th = rng.normal(0, 0.3, nparam)
    X = rng.normal(0, 1, (B, F))
    Y = np.stack([rng.integers(0, h, B) for h in HEADS], axis=1)
    return th, X, Y


def test_forward_matches_oracle(llp):
    th, X, _ = rand_problem(1)
    d = llp.mlp_dims()
    z = llp.mlp_forward(d, torch.tensor(th, dtype=torch.float32, device="cuda"),
                        torch.tensor(X, dtype=torch.float32, device="cuda")).cpu().numpy()
    zr, _ = omlp.forward(th.astype(np.float32).astype(np.float64), X.astype(np.float32).astype(np.float64), F, H1, H2, O)
    assert np.allclose(z, zr, rtol=1e-4, atol=1e-4 * np.abs(zr).max())


@pytest.mark.parametrize("seed", [2, 3])
def test_loss_and_gradient_match_oracle(llp, seed):
    th, X, Y = rand_problem(seed)
    th32 = th.astype(np.float32)
    X32 = X.astype(np.float32)
    d = llp.mlp_dims()
    loss, grad, _ = llp.mlp_loss_grad(d, torch.tensor(th32, device="cuda"), torch.tensor(X32, device="cuda"),
                                      torch.tensor(Y, dtype=torch.int32, device="cuda"))
    Lr, gr = omlp.backward(th32.astype(np.float64), X32.astype(np.float64), Y, HEADS, F, H1, H2, O)
    assert abs(float(loss.item()) - Lr) <= 1e-4 * max(1.0, abs(Lr))
    g = grad.cpu().numpy()
    assert np.allclose(g, gr, rtol=1e-3, atol=1e-4 * np.abs(gr).max())


def test_adam_step_matches_oracle(llp):
    rng = np.random.default_rng(4)
    p = rng.normal(0, 1, 1000).astype(np.float32)
    g = rng.normal(0, 1, 1000).astype(np.float32)
    m = rng.normal(0, 0.1, 1000).astype(np.float32)
    v = rng.uniform(0, 0.1, 1000).astype(np.float32)
    tp, tg, tm, tv = (torch.tensor(a, device="cuda") for a in (p, g, m, v))
    llp.mlp_adam(tp, tg, tm, tv, 7, 1e-3)
    rp, rm, rv = omlp.adam_step(p.astype(np.float64), g.astype(np.float64), m.astype(np.float64),
                                v.astype(np.float64), 7, 1e-3)
    assert np.allclose(tp.cpu().numpy(), rp, rtol=1e-5, atol=1e-6)
    assert np.allclose(tm.cpu().numpy(), rm, rtol=1e-5, atol=1e-7)
    assert np.allclose(tv.cpu().numpy(), rv, rtol=1e-5, atol=1e-8)


def test_training_reduces_loss(llp):
    from paper_2603_13147_b300 import sched
    rng = np.random.default_rng(5)
    X = rng.normal(0, 1, (64, F)).astype(np.float32)
    Y = np.stack([(X[:, 0] > 0).astype(int), (X[:, 1] > 0).astype(int) * 3, (X[:, 2] > 0).astype(int),
                  (X[:, 3] > 0).astype(int) * 2, (X[:, 4] > 0).astype(int) * 4], 1)
    params, hist = sched.train(X, Y.astype(np.int32), steps=400, lr=1e-2)
    assert hist[-1][1] < 0.5 * hist[0][1]
    assert (sched.predict(params, X) == Y).mean() > 0.9


def test_device_inference_matches_oracle_network(llp):
    """The on-device feature + inference kernels pick the oracle network's argmax."""
    from paper_2603_13147_b300 import sched
    g = synth.rmat(14, seed=8)
    s = synth.max_out_degree_vertex(g)
    dg = llp.DeviceGraph.from_host(g, "cuda")
    for seed in range(6):
        th = sched.init_params(seed)
        chosen, feats = llp.graph_schedule(dg, s, torch.tensor(th, device="cuda"))
        assert abs(feats[0] - np.log2(g["n"] + 1)) < 1e-4 and abs(feats[1] - np.log2(g["m"] + 1)) < 1e-4
        z, _ = omlp.forward(th.astype(np.float64), np.array([feats], np.float64), F, H1, H2, O)
        z = z[0]
        pred = [int(np.argmax(z[0:3])), int(np.argmax(z[3:11])), int(np.argmax(z[11:14])),
                int(np.argmax(z[14:18])), int(np.argmax(z[18:23]))]
        assert chosen.mode == pred[0]
        assert chosen.block_cfg == pred[2] + 1
        assert chosen.local_chain == sched.CHAIN_OF_CLASS[pred[3]]
        assert chosen.group_words == sched.GW_OF_CLASS[pred[4]]
        want = sched.delta_of_class(pred[1], sched.sampled_wmax(g))
        assert chosen.delta == want


@pytest.mark.parametrize("seed", range(8))
def test_results_bit_exact_under_any_learned_schedule(llp, seed):
    """Random networks make arbitrary choices; every result stays identical to the oracle's."""
    from paper_2603_13147_b300 import sched
    gs = [(synth.er16k(), 0), (synth.rmat(15, seed=3), None), (synth.grid_graph(48, 48, 1, 1000, seed=4), 0)]
    th = torch.tensor(sched.init_params(100 + seed) * 3.0, device="cuda")
    for g, s in gs:
        s = synth.max_out_degree_vertex(g) if s is None else s
        dg = llp.DeviceGraph.from_host(g, "cuda")
        d, ws = llp.sssp(dg, s, sched=llp.make_sched(use_mlp=1, mlp_params=th))
        st = llp.get_status(ws)
        assert st["status"] == 0
        assert (llp.as_u32(d) == oracle.sssp(g["offsets"], g["indices"], g["weights"], s)).all()
        lv, ws = llp.bfs(dg, s, sched=llp.make_sched(use_mlp=1, mlp_params=th), ws=ws)
        assert (llp.as_u32(lv) == oracle.bfs(g["offsets"], g["indices"], s)).all()


def test_trained_model_loads_and_schedules(llp):
    from paper_2603_13147_b300 import sched
    if not os.path.exists(sched.MODEL_PATH):
        pytest.skip("no trained scheduler model in the package")
    p = sched.load_model()
    assert p.numel() == llp.mlp_param_count(llp.mlp_dims())
    g = synth.grid_graph(64, 64, 1, 1000, seed=2)
    dg = llp.DeviceGraph.from_host(g, "cuda")
    d, ws = llp.sssp(dg, 0, sched=sched.learned_sched(p))
    assert (llp.as_u32(d) == oracle.sssp(g["offsets"], g["indices"], g["weights"], 0)).all()


@pytest.mark.parametrize("seed", range(4))
def test_learned_prologue_with_warm_start_pull_and_int64(llp, seed):
    """The learned run's prologue initialises the state (keeping a warm start's distances), and
    the sweep rebuilds the class table when the chosen block configuration moves the degree limit:
    warm starts, BFS with pull sweeps and int64 offsets stay identical to the oracle under random
    networks."""
    from paper_2603_13147_b300 import sched
    th = torch.tensor(sched.init_params(200 + seed) * 3.0, device="cuda")
    learned = llp.make_sched(use_mlp=1, mlp_params=th)
    g = synth.rmat(14, seed=20 + seed)
    s = synth.max_out_degree_vertex(g)
    ref = oracle.sssp(g["offsets"], g["indices"], g["weights"], s)
    # warm start: the oracle result of slightly heavier weights, then the true weights
    w_up = g["weights"].copy()
    w_up[::7] += 5
    prev = oracle.sssp(g["offsets"], g["indices"], w_up, s)
    dg = llp.DeviceGraph.from_host(g, "cuda")
    dist = torch.from_numpy(prev.view(np.int32).copy()).cuda()
    seeds = torch.from_numpy(np.unique(np.searchsorted(g["offsets"], np.arange(0, g["m"], 7), side="right") - 1)
                             .astype(np.int32)).cuda()
    d, ws = llp.sssp_warm(dg, s, dist, seeds, sched=learned)
    assert llp.get_status(ws)["status"] == 0
    assert (llp.as_u32(d) == ref).all()
    # BFS with pull sweeps over the device transpose
    lv, ws = llp.bfs_pull(dg, dg.transpose(), s, sched=learned, ws=ws)
    assert (llp.as_u32(lv) == oracle.bfs(g["offsets"], g["indices"], s)).all()
    # int64 offsets
    d64, ws = llp.sssp(llp.DeviceGraph.from_host(g, "cuda", offsets_64=True), s, sched=learned, ws=ws)
    assert (llp.as_u32(d64) == ref).all()
