"""What the trained scheduler network gains over the fixed heuristic schedule, on
held-out graphs (sizes and seeds not in its training set).  Results must be
identical; the learned schedule must not be slower in total."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _time(fn, reps=3):
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


def test_learned_schedule_gain_on_held_out_graphs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2603_13147_b300 as llp
    from paper_2603_13147_b300 import sched
    import os
    if not os.path.exists(sched.MODEL_PATH):
        pytest.skip("no trained scheduler model in the package")
    params = sched.load_model()
    learned = sched.learned_sched(params)
    items = [("grid1536", synth.grid_graph(1536, 1536, 1, 1000, seed=77), 0),
             ("rmat19", synth.rmat(19, seed=78), None),
             ("er19_d8", synth.er_graph(1 << 19, 8 << 19, 1, 100, seed=79), 0)]
    tot_h = tot_l = 0.0
    report = {}
    for name, g, s in items:
        s = synth.max_out_degree_vertex(g) if s is None else s
        dg = llp.DeviceGraph.from_host(g, "cuda")
        ws = llp.workspace(llp.sssp_workspace_size(g["n"], g["m"]))
        out = torch.empty(g["n"], dtype=torch.int32, device="cuda")
        th = _time(lambda: llp.sssp(dg, s, out=out, ws=ws))
        ref = oracle.sssp(g["offsets"], g["indices"], g["weights"], s)
        assert (llp.as_u32(out) == ref).all()
        tl = _time(lambda: llp.sssp(dg, s, out=out, ws=ws, sched=learned))
        st = llp.get_status(ws)
        assert st["status"] == 0 and (llp.as_u32(out) == ref).all()
        report[name] = (round(th, 3), round(tl, 3), st["mode_used"], st["delta_used"], st["block_cfg_used"],
                        st["local_chain_used"])
        tot_h += th
        tot_l += tl
    print("heuristic ms, learned ms, learned schedule:", report, "total gain", tot_h / tot_l)
    assert tot_l < tot_h
