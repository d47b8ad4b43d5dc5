"""Learned scheduler of the graph sweep: training data, training, model file.

The network (features -> 64 -> 64 -> {mode, bucket-width class, block_cfg,
local-chain class, dense-sweep group-width class})
runs on the device inside llp_sssp / llp_bfs when llp_sched_t.use_mlp = 1.
Training data are timings of the plain engine: for each generated graph, the
schedule space is searched coordinate-wise (bucket width, mode, local chain,
block configuration, group width; each candidate timed with CUDA events, median
of 3), and
the fastest schedule becomes the label.  The features come from the same device
feature kernel the engine uses at run time.  Training is full-batch Adam with
the library's own fp32 forward/backward/Adam kernels.  The schedule never
changes results, only time.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np
import torch

from . import binding as B

MODEL_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sched_model.npz")
N_DELTA_CLASSES = SCHED_DELTA = 8


def sampled_wmax(g: dict) -> int:
    """Largest arc weight over the same evenly spaced sample the device feature kernel uses."""
    w = g.get("weights")
    m = int(g["m"])
    if w is None or m == 0:
        return 1
    S = min(m, 16384)
    e = (np.arange(S, dtype=np.int64) * m) // S
    return int(w[e].max())


def delta_of_class(c: int, wmax: int) -> int:
    """Bucket width of class c (0 = no buckets), as the inference kernel maps it."""
    if c == 0:
        return B.DELTA_INF
    wd = float(np.float32(wmax)) * 2.0 ** (c - 1)
    return 1 if wd < 1.0 else int(min(wd, 2147483647.0))


def _time_call(fn, reps=3, cap_ms=None):
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
        if cap_ms is not None and ts[-1] > cap_ms:
            break
    return float(np.median(ts))


CHAIN_OF_CLASS = (0, 4, 16, 64)
GW_OF_CLASS = (0, 1, 2, 4, 8)  # 0: the engine's grid-size rule


def label_graph(dg: B.DeviceGraph, source: int, unit: bool, wmax: int, ws=None, passes: int = 2,
                margin: float = 0.03, reps: int = 3):
    """Coordinate search over (mode, bucket class, block class, chain class, group-width class),
    starting from the heuristic default; a coordinate moves only when a candidate is faster by more
    than `margin`.
    Returns (label tuple of class indices, timing log, best ms)."""
    if ws is None:
        ws = B.workspace(B.sssp_workspace_size(dg.n, dg.m), dg.indices.device)
    out = torch.empty(dg.n, dtype=torch.int32, device=dg.indices.device)
    fn = B.bfs if unit else B.sssp
    log = {}

    def run(lab, cap):
        key = ",".join(map(str, lab))
        if key in log:
            return log[key]
        s = B.make_sched(mode=lab[0], delta=delta_of_class(lab[1], wmax), block_cfg=lab[2] + 1,
                         local_chain=CHAIN_OF_CLASS[lab[3]] if lab[3] else -1, group_words=GW_OF_CLASS[lab[4]])
        t = _time_call(lambda: fn(dg, source, out=out, sched=s, ws=ws), reps=reps, cap_ms=cap)
        log[key] = t
        return t

    best = [0, 0, 1, 0, 0]  # AUTO, no buckets, block cfg 2, no chain, group-width rule: the heuristic
    best_t = run(best, None)
    axes = [(1, [0] if unit else list(range(N_DELTA_CLASSES))), (0, [0, 1, 2]), (3, [0, 1, 2, 3]), (2, [0, 1, 2]),
            (4, [0, 1, 2, 3, 4])]
    for _ in range(passes):
        moved = False
        for ax, vals in axes:
            for val in vals:
                if val == best[ax]:
                    continue
                cand = list(best)
                cand[ax] = val
                t = run(cand, 20 * best_t)
                if t < best_t * (1.0 - margin):
                    best_t, best, moved = t, cand, True
        if not moved:
            break
    return tuple(best), log, best_t


def label_to_sched(label, wmax: int) -> B.Sched:
    """Class tuple (mode, bucket class, block class 0..2, chain class 0..3, group-width class 0..4) ->
    schedule."""
    return B.make_sched(mode=int(label[0]), delta=delta_of_class(int(label[1]), wmax), block_cfg=int(label[2]) + 1,
                        local_chain=CHAIN_OF_CLASS[int(label[3])] if int(label[3]) else -1,
                        group_words=GW_OF_CLASS[int(label[4])])


def training_graphs(seed: int = 11, quick: bool = False):
    """Generated training instances: power-law (R-MAT), road-like (grids), uniform (ER); SSSP and BFS."""
    import synth
    rng = np.random.default_rng(seed)
    items = []
    scales = [14, 16, 18] if quick else [14, 15, 16, 17, 18, 19, 20]
    for sc in scales:
        for ef, (wlo, whi) in ((16, (1, 255)), (8, (1, 1000)), (16, (1, 10))):
            g = synth.rmat_graph(sc, ef, 0.57, 0.19, 0.19, wlo, whi, seed=int(rng.integers(1 << 30)))
            items.append((f"rmat{sc}_ef{ef}_w{whi}", g, synth.max_out_degree_vertex(g), False))
        g = synth.rmat_graph(sc, 16, 0.45, 0.22, 0.22, 1, 255, seed=int(rng.integers(1 << 30)))
        items.append((f"rmat{sc}_flat", g, synth.max_out_degree_vertex(g), False))
        items.append((f"rmat{sc}_bfs", g, synth.max_out_degree_vertex(g), True))
    if not quick:
        # larger power-law instances (block configuration and group width matter more there)
        for sc in (21, 22, 23, 24):
            g = synth.rmat_graph(sc, 16, 0.57, 0.19, 0.19, 1, 255, seed=int(rng.integers(1 << 30)))
            items.append((f"rmat{sc}_ef16_w255", g, synth.max_out_degree_vertex(g), False))
    sides = [64, 128, 256] if quick else [64, 128, 256, 384, 512, 768, 1024, 1280, 1536, 2048]
    for side in sides:
        for whi in (1000, 100):
            g = synth.grid_graph(side, side, 1, whi, seed=int(rng.integers(1 << 30)))
            items.append((f"grid{side}_w{whi}", g, 0, False))
        items.append((f"grid{side}_bfs", g, 0, True))
    for lg in ([14, 17] if quick else [14, 16, 18, 20]):
        for deg in (4, 16):
            n = 1 << lg
            g = synth.er_graph(n, n * deg, 1, 100, seed=int(rng.integers(1 << 30)))
            items.append((f"er{lg}_d{deg}", g, 0, False))
    return items


def collect(items, device="cuda", verbose=True):
    """Features (device kernel) and timing labels for every training item."""
    X, Y, meta = [], [], []
    dummy = torch.zeros(B.mlp_param_count(B.mlp_dims()), dtype=torch.float32, device=device)
    for name, g, src, unit in items:
        dg = B.DeviceGraph.from_host(g, device)
        _, feats = B.graph_schedule(dg, src, dummy, unit_weights=unit)
        wmax = sampled_wmax(g) if not unit else 1
        t0 = time.time()
        # training labels move off the default only for a clear gain (timing noise is ~2 %)
        label, log, best_ms = label_graph(dg, src, unit, wmax, margin=0.05, reps=5)
        X.append(feats)
        Y.append(list(label))
        meta.append({"name": name, "label": label, "best_ms": best_ms, "log": log, "wall_s": time.time() - t0})
        if verbose:
            print(json.dumps({"name": name, "label": label, "best_ms": round(best_ms, 4)}), flush=True)
        del dg
    return np.array(X, np.float32), np.array(Y, np.int32), meta


def init_params(seed: int = 0, d=None) -> np.ndarray:
    d = d or B.mlp_dims()
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, fan_out in ((d.F, d.H1), (d.H1, d.H2), (d.H2, d.O)):
        parts.append(rng.normal(0, np.sqrt(2.0 / fan_in), (fan_in, fan_out)).ravel())
        parts.append(np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)


def train(X: np.ndarray, Y: np.ndarray, steps: int = 3000, lr: float = 3e-3, seed: int = 0, device="cuda",
          verbose=False):
    """Full-batch Adam with the library's kernels.  Returns (params tensor, loss history)."""
    d = B.mlp_dims()
    p = torch.from_numpy(init_params(seed, d)).to(device)
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    Xd = torch.from_numpy(np.ascontiguousarray(X, np.float32)).to(device)
    Yd = torch.from_numpy(np.ascontiguousarray(Y, np.int32)).to(device)
    hist = []
    ws = None
    for t in range(1, steps + 1):
        loss, grad, ws = B.mlp_loss_grad(d, p, Xd, Yd, ws=ws)
        B.mlp_adam(p, grad, m, v, t, lr)
        if t % 100 == 0 or t == 1:
            hist.append((t, float(loss.item())))
            if verbose:
                print("step", t, hist[-1][1], flush=True)
    return p, hist


def predict(params: torch.Tensor, X: np.ndarray) -> np.ndarray:
    d = B.mlp_dims()
    z = B.mlp_forward(d, params, torch.from_numpy(np.ascontiguousarray(X, np.float32)).to(params.device))
    z = z.cpu().numpy()
    out, lo = [], 0
    for h in B.SCHED_HEADS:
        out.append(z[:, lo:lo + h].argmax(axis=1))
        lo += h
    return np.stack(out, axis=1)


def save_model(params: torch.Tensor, path: str = MODEL_PATH, meta=None):
    np.savez(path, params=params.detach().cpu().numpy().astype(np.float32),
             meta=json.dumps(meta or {}))


def load_model(path: str = MODEL_PATH, device="cuda") -> torch.Tensor:
    """The trained parameters; refuses a file whose size does not match the network's shape
    (the device kernels read exactly that many parameters)."""
    z = np.load(path)
    want = B.mlp_param_count(B.mlp_dims())
    if z["params"].size != want:
        raise ValueError(f"scheduler model {path} has {z['params'].size} parameters, the network needs {want}")
    return torch.from_numpy(z["params"].astype(np.float32)).to(device)


def learned_sched(params: torch.Tensor) -> B.Sched:
    return B.make_sched(use_mlp=1, mlp_params=params)


if __name__ == "__main__":
    import argparse
    import sys
    ap = argparse.ArgumentParser(description="collect timing labels and train the scheduler network")
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--out", default=MODEL_PATH)
    ap.add_argument("--data-out", default=None)
    ap.add_argument("--steps", type=int, default=3000)
    a = ap.parse_args()
    items = training_graphs(quick=a.quick)
    X, Y, meta = collect(items)
    params, hist = train(X, Y, steps=a.steps, verbose=True)
    acc = (predict(params, X) == Y).mean(axis=0).tolist()
    save_model(params, a.out, {"items": [mm["name"] for mm in meta], "labels": Y.tolist(), "train_acc": acc,
                               "loss": hist})
    if a.data_out:
        np.savez(a.data_out, X=X, Y=Y, meta=json.dumps(meta))
    print(json.dumps({"train_acc_per_head": acc, "final_loss": hist[-1][1], "n": len(items)}))
    sys.exit(0)
