"""Benchmark: LLP-SSSP (and LLP-BFS) on an R-MAT scale-22 graph on one B300.

One step = one llp_sssp call (the whole forbidden/advance sweep to the fixed
point: init, worklist sweeps, bucket handling, termination, output) on the
R-MAT scale 22, edge factor 16 graph (4,194,304 vertices, 67,108,864 arcs,
weights U[1,255], source = highest out-degree vertex), inputs resident in HBM.
`value` = GTEPS = arcs of reached vertices / step time (whole job: summed over
ranks, divided by the max time over ranks).  The L2 is flushed between timed
steps (a 256 MB write), and the CSR (537 MB) is larger than the L2 anyway.

--impl reference times the sequential CPU oracle (Dijkstra) on the host cores
instead, on the same graph, as the reference arm.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SCALE = 22
WORKLOAD = "rmat22_ef16_sssp"

# DRAM traffic of the sweep kernel per algorithmic byte, from one ncu capture at
# R-MAT scale 20 (dram__bytes_read.sum + dram__bytes_write.sum of one launch), valid
# only for the kernel source it was taken from (sha256 prefix of graph_sweep.cu +
# llp_common.cuh).
TRAFFIC_CAPTURE = {"src_sha": "8a0ed638958a5a85", "bytes_per_alg_byte": 1.2817}


def kernel_src_sha():
    import hashlib
    h = hashlib.sha256()
    for f in ("graph_sweep.cu", "llp_common.cuh"):
        with open(os.path.join(ROOT, "paper_2603_13147_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """Samples the SM clock, its maximum and the clock-event (throttle) reasons while
    running: through NVML in this process every ~0.2 ms plus the query time (the
    timed regions are a few milliseconds long), else through nvidia-smi every 200 ms.  Only samples taken
    between __enter__ and __exit__ are kept."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    # NVML clock-event reason bits (nvml.h, nvmlClocksEventReason*)
    REASON_BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20,
                   "hw_thermal_slowdown": 0x40}

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []  # (sm_mhz, max_mhz, {reason: bool})
        self.source = None
        self._stop = threading.Event()
        self._t = None
        self._nvml = None
        try:
            self._nvml = self._nvml_open()
            self.source = "nvml"
        except Exception:
            self._nvml = None
            self.source = "nvidia-smi"

    def _nvml_open(self):
        """NVML through its C API (libnvidia-ml, shipped with the driver): (library, handle)
        of CUDA device `gpu`, found through the visible-device list (index or UUID)."""
        nv = ctypes.CDLL("libnvidia-ml.so.1")
        if nv.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        hd = ctypes.c_void_p()
        ids = [x.strip() for x in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if x.strip()]
        if ids and self.gpu < len(ids) and not ids[self.gpu].isdigit():
            rc = nv.nvmlDeviceGetHandleByUUID(ids[self.gpu].encode(), ctypes.byref(hd))
        else:
            idx = int(ids[self.gpu]) if ids and self.gpu < len(ids) else self.gpu
            rc = nv.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(idx), ctypes.byref(hd))
        if rc != 0:
            raise RuntimeError("no NVML handle")
        reasons = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            nv.nvmlDeviceGetCurrentClocksThrottleReasons
        return nv, hd, reasons

    def _sample_nvml(self):
        nv, hd, reasons = self._nvml
        sm, mx, bits = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
        if (nv.nvmlDeviceGetClockInfo(hd, 1, ctypes.byref(sm)) != 0 or  # 1 = NVML_CLOCK_SM
                nv.nvmlDeviceGetMaxClockInfo(hd, 1, ctypes.byref(mx)) != 0 or reasons(hd, ctypes.byref(bits)) != 0):
            return
        self.rows.append((float(sm.value), float(mx.value),
                          {k: bool(bits.value & b) for k, b in self.REASON_BITS.items()}))

    def _sample_smi(self):
        out = subprocess.run(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                              "-i", str(self.gpu)], capture_output=True, text=True, timeout=5).stdout
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            r = [x.strip() for x in line.split(",")]
            if len(r) >= 9 and r[1].replace('.', '', 1).isdigit() and r[2].replace('.', '', 1).isdigit():
                self.rows.append((float(r[1]), float(r[2]),
                                  {nm: r[5 + i].lower().startswith("active") for i, nm in enumerate(names)}))

    def _run(self):
        while not self._stop.is_set():
            try:
                if self._nvml:
                    self._sample_nvml()
                else:
                    self._sample_smi()
            except Exception:
                pass
            self._stop.wait(0.0002 if self._nvml else 0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self._t:
            self._t.join(timeout=10)

    def summary(self):
        sm = [r[0] for r in self.rows]
        mx = [r[1] for r in self.rows]
        reasons = sorted({k for r in self.rows for k, on in r[2].items() if on})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows), "source": self.source}


def combine_ranks(ms_local: float, units_local: int, device=None):
    """Whole-job numbers over the process group: the max step time over ranks and the
    units processed by all ranks (summed).  Single-process: the local values."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return ms_local, units_local
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    u = torch.tensor([units_local], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), int(u.item())


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def make_graph(scale=SCALE):
    import synth
    g = synth.rmat(scale)
    s = synth.max_out_degree_vertex(g)
    return g, s


def cpu_info():
    """Host cores this process may use and the CPU model (for every cpu_baseline)."""
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    model = "unknown"
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return cores, model


def cpu_time(fn):
    t = time.perf_counter()
    r = fn()
    return time.perf_counter() - t, r


def oracle_parallel(tasks, threads):
    """Runs independent oracle calls (closures) on `threads` host threads (the oracle's C code
    runs outside the GIL) and returns the wall time."""
    import concurrent.futures as cf
    t = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        for f in [ex.submit(fn) for fn in tasks]:
            f.result()
    return time.perf_counter() - t


def reached_arcs(g, dist_u32):
    deg = np.diff(g["offsets"])
    reached = dist_u32 != 0xFFFFFFFF
    return int(deg[reached].sum()), int(reached.sum())


def cpu_oracle_sample(g, s, budget_s=20.0):
    """Times the oracle (Dijkstra, one host core) on the full graph; returns (GTEPS, seconds, dist)."""
    import oracle
    t = time.perf_counter()
    d = oracle.sssp(g["offsets"], g["indices"], g["weights"], s)
    dt = time.perf_counter() - t
    mr, _ = reached_arcs(g, d)
    return mr / dt / 1e9, dt, d


def oracle_bfs_levels(g, s):
    import oracle
    return oracle.bfs(g["offsets"], g["indices"], s)


def oracle_sssp_w(g, w, s):
    import oracle
    return oracle.sssp(g["offsets"], g["indices"], w, s)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    g, s = make_graph()
    times = []
    mr = None
    for i in range(args.warmup + args.steps):
        g_teps, dt, d = cpu_oracle_sample(g, s)
        if mr is None:
            mr, _ = reached_arcs(g, d)
        if i >= args.warmup:
            times.append(dt)
    t = float(np.mean(times))
    v = mr / t / 1e9
    line = {"impl": "reference", "metric": "SSSP GTEPS (R-MAT scale 22, ef 16)", "value": v, "unit": "GTEPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "config": {"workload": WORKLOAD if args.scale == SCALE else f"rmat{args.scale}_ef16_sssp", "n": g.n, "m": g.m, "source": s},
            "cpu_baseline": {"value": v, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                             "sample": "full graph, one Dijkstra (binary heap) per step on one host core"},
            "e2e": {"value": v, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args):
    import torch
    import paper_2603_13147_b300 as llp

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    llp.lib()

    g, s = make_graph(args.scale)
    dg = llp.DeviceGraph.from_host(g, dev)
    ws = llp.workspace(llp.sssp_workspace_size(g.n, g.m), dev)
    dist_t = torch.empty(g.n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    sched = None

    clocks = ClockSampler(dev.index if dev.index is not None else 0)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    # warm-up (also checks the device status), directly followed by the timed steps so
    # that the GPU does not idle in between
    for i in range(args.warmup):
        flush.fill_(i & 0xFF)
        llp.sssp(dg, s, out=dist_t, sched=sched, ws=ws)
    st = llp.get_status(ws)
    if st["status"] != 0:
        raise RuntimeError(f"llp_sssp device status {st}")

    # timed region: per-step CUDA events on the launching stream, L2 flushed between steps
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    with clocks:
        t_wall0 = time.perf_counter()
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            ev[i][0].record(stream)
            llp.sssp(dg, s, out=dist_t, sched=sched, ws=ws)
            ev[i][1].record(stream)
        torch.cuda.synchronize(dev)
        t_wall = time.perf_counter() - t_wall0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = float(np.mean(step_ms))
    st = llp.get_status(ws)
    if st["status"] != 0:
        raise RuntimeError(f"llp_sssp device status {st}")
    d_host = llp.as_u32(dist_t)
    mr, nr = reached_arcs(g, d_host)
    slog = llp.sweep_log(ws)
    ms, units = combine_ranks(ms, mr, device=dev)
    value = units / (ms * 1e-3) / 1e9

    # roofline of the sweep kernel: algorithmic bytes 8*m_r (index + weight per
    # arc of a reached vertex) + 8*n (offsets pair / distance per vertex)
    alg_bytes = 8 * mr + 8 * g.n
    peak, peak_kind = peaks()
    achieved = alg_bytes / (ms * 1e-3) / 1e9
    traffic = None
    if kernel_src_sha() == TRAFFIC_CAPTURE["src_sha"]:
        traffic = int(TRAFFIC_CAPTURE["bytes_per_alg_byte"] * alg_bytes)

    # access-pattern floor of a push sweep on this graph: one pass over all m arcs, CSR
    # streamed, one random read of per-vertex state per arc (llp_gather_floor), same protocol
    sink = llp.gather_floor(dg, dist_t)
    torch.cuda.synchronize(dev)
    fev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        fev[i][0].record(stream)
        llp.gather_floor(dg, dist_t, sink=sink)
        fev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    floor_ms = float(np.mean([a.elapsed_time(b) for a, b in fev]))
    del sink

    # BFS on the same graph (reported beside the headline)
    for _ in range(2):
        llp.bfs(dg, s, out=dist_t, ws=ws)
    torch.cuda.synchronize(dev)
    bev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        bev[i][0].record(stream)
        llp.bfs(dg, s, out=dist_t, ws=ws)
        bev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    bfs_ms = float(np.mean([a.elapsed_time(b) for a, b in bev]))
    bfs_st = llp.get_status(ws)
    bfs_lv = llp.as_u32(dist_t)
    bfs_mr, _ = reached_arcs(g, bfs_lv)

    # BFS with pull sweeps over the device transpose (built once, outside the timed steps)
    torch.cuda.synchronize(dev)
    tt0 = torch.cuda.Event(enable_timing=True); tt1 = torch.cuda.Event(enable_timing=True)
    tt0.record(stream)
    dg_in = dg.transpose()
    tt1.record(stream)
    for _ in range(2):
        llp.bfs_pull(dg, dg_in, s, out=dist_t, ws=ws)
    torch.cuda.synchronize(dev)
    transpose_ms = tt0.elapsed_time(tt1)
    pev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        pev[i][0].record(stream)
        llp.bfs_pull(dg, dg_in, s, out=dist_t, ws=ws)
        pev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    pull_ms = float(np.mean([a.elapsed_time(b) for a, b in pev]))
    pull_st = llp.get_status(ws)
    pull_lv = llp.as_u32(dist_t)
    pull_same = bool((pull_lv == bfs_lv).all())
    del dg_in

    # warm start: 0.1 % of the arc weights decreased (w -> max(1, w // 3)); re-solve from the
    # previous distances with the tails of those arcs as seeds, against a cold solve
    rng = np.random.default_rng(77)
    dec = np.sort(rng.choice(g.m, g.m // 1000, replace=False))
    w2 = g["weights"].copy()
    w2[dec] = np.maximum(1, w2[dec] // 3)
    seeds = np.unique(np.searchsorted(g["offsets"], dec, side="right") - 1).astype(np.int32)
    dg2 = llp.DeviceGraph(dg.offsets, dg.indices, torch.from_numpy(w2.view(np.int32)).to(dev))
    seeds_t = torch.from_numpy(seeds).to(dev)
    d_old = torch.from_numpy(d_host.view(np.int32)).to(dev)
    d_warm = torch.empty_like(d_old)
    cold_t, warm_t = [], []
    for i in range(args.steps + 1):
        for warm in (False, True):
            if warm:
                d_warm.copy_(d_old)
            flush.fill_(i & 0xFF)
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if warm:
                llp.sssp_warm(dg2, s, d_warm, seeds_t, ws=ws)
            else:
                llp.sssp(dg2, s, out=dist_t, ws=ws)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            if i > 0:
                (warm_t if warm else cold_t).append(e0.elapsed_time(e1))
    warm_st = llp.get_status(ws)
    warm_same = bool(torch.equal(d_warm, dist_t))
    d_warm_host = llp.as_u32(d_warm)
    w2_host = w2
    del dg2

    # end to end through the C ABI with HOST buffers (llp_sssp_host): every step copies the graph
    # from pinned host memory into a workspace, sweeps, and copies the distances back; steps
    # alternate between two streams and workspaces, so a step's copies overlap the previous
    # step's sweep (the host-to-device link is the bound)
    import numpy as _np
    h_off = torch.from_numpy(g["offsets"].astype(_np.int32)).pin_memory()
    h_idx = torch.from_numpy(g["indices"]).pin_memory()
    h_w = torch.from_numpy(g["weights"].view(_np.int32)).pin_memory()
    h_outs = [torch.empty(g.n, dtype=torch.int32).pin_memory() for _ in range(2)]
    ws_hs = [llp.workspace(llp.sssp_host_workspace_size(g.n, g.m), dev) for _ in range(2)]
    sts = [stream, torch.cuda.Stream(dev)]
    for j in range(2):  # warm-up, one step per stream
        llp.sssp_host(h_off, h_idx, h_w, s, h_outs[j], ws=ws_hs[j], stream=sts[j])
    torch.cuda.synchronize(dev)
    e2e_steps = max(2, min(args.steps, 5))
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(sts[0])
    sts[1].wait_event(e0)
    for i in range(e2e_steps):
        j = i % 2
        llp.sssp_host(h_off, h_idx, h_w, s, h_outs[j], ws=ws_hs[j], stream=sts[j])
    join = torch.cuda.Event()
    join.record(sts[1])
    sts[0].wait_event(join)
    e1.record(sts[0])
    torch.cuda.synchronize(dev)
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    e2e_same = all(bool((h.numpy().view(_np.uint32) == d_host).all()) for h in h_outs)
    h_out = h_outs[0]
    del ws_hs
    h2d = h_off.numel() * 4 + h_idx.numel() * 4 + h_w.numel() * 4
    d2h = h_out.numel() * 4

    line = {
        "metric": "SSSP GTEPS (R-MAT scale 22, ef 16)", "value": value, "unit": "GTEPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD if args.scale == SCALE else f"rmat{args.scale}_ef16_sssp", "n": g.n, "m": g.m, "source": s, "reached_vertices": nr,
                   "reached_arcs": mr, "l2": "flushed between steps (256 MB write); CSR 537 MB > L2",
                   "parallelism": "replicas" if world > 1 else "single-gpu",
                   "schedule": {k: st[k] for k in ("mode_used", "delta_used", "block_cfg_used")}},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "traffic_note": "scaled from an R-MAT scale 20 capture by algorithmic bytes", "peak_kind": peak_kind, "frac_of_nominal_8tbs": achieved / 8000.0,
                     "alg_bytes_per_launch": alg_bytes, "kernel": "graph_sweep_kernel<int32,false>",
                     "gather_floor_ms": floor_ms,
                     "gather_floor_note": "llp_gather_floor: one pass over all m arcs, CSR streamed with 16-byte "
                                          "loads, one random read of per-vertex state per arc, 8 in flight per lane",
                     "gather_floor_g_arcs_per_s": g.m / (floor_ms * 1e-3) / 1e9,
                     "sweep_g_arcs_per_s": st["edges"] / (ms * 1e-3) / 1e9,
                     "floor_for_arcs_examined_ms": floor_ms * st["edges"] / g.m},
        "sweep_stats": {"sweeps": st["sweeps"], "edges_scanned": st["edges"], "advances": st["advances"],
                        "dense_sweeps": st["dense_sweeps"], "edges_per_reached_arc": st["edges"] / max(mr, 1),
                        "device_loop_ms": st["elapsed_ns"] / 1e6,
                        "step_ms_min_median_max": [float(np.min(step_ms)), float(np.median(step_ms)),
                                                   float(np.max(step_ms))],
                        "per_sweep": [[round(int(r[0]) / 1e6, 4), int(r[1]), int(r[2]), int(r[3])] for r in slog]},
        "bfs": {"gteps": bfs_mr / (bfs_ms * 1e-3) / 1e9, "ms": bfs_ms, "sweeps": bfs_st["sweeps"],
                "edges_scanned": bfs_st["edges"], "status": bfs_st["status"],
                "pull": {"gteps": bfs_mr / (pull_ms * 1e-3) / 1e9, "ms": pull_ms, "sweeps": pull_st["sweeps"],
                         "pull_sweeps": pull_st["pull_sweeps"], "edges_scanned": pull_st["edges"],
                         "status": pull_st["status"], "levels_equal_push": pull_same,
                         "transpose_ms": transpose_ms,
                         "note": "llp_bfs_pull with the device transpose (built once, untimed); "
                                 "GTEPS counts the reached arcs, as for push"}},
        "warm_start": {"changed_arcs": int(len(dec)), "seeds": int(len(seeds)),
                       "cold_ms": float(np.mean(cold_t)), "warm_ms": float(np.mean(warm_t)),
                       "speedup": float(np.mean(cold_t) / np.mean(warm_t)), "warm_sweeps": warm_st["sweeps"],
                       "warm_edges_scanned": warm_st["edges"], "equals_cold": warm_same,
                       "note": "llp_sssp_warm from the previous distances after 0.1% of the weights "
                               "decreased; dist copy outside the timed region"},
        "e2e": {"value": mr / (e2e_ms * 1e-3) / 1e9, "unit": "GTEPS", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                "call": "llp_sssp_host (pinned host CSR), steps alternating over two streams",
                "result_equals_device_run": e2e_same},
        "gpu_launches": args.steps,
        "clocks": clocks.summary(),
        "wall_s_timed": t_wall,
    }
    cpu = rank == 0 and not args.no_cpu_baseline
    dt22 = None
    if cpu:
        gt, dt22, dref = cpu_oracle_sample(g, s)
        cores, model = cpu_info()
        line["cpu_baseline"] = {"value": gt, "unit": "GTEPS", "cores": 1, "cpu_model": model,
                                "host_cores": cores, "kind": "oracle",
                                "sample": f"full graph, one Dijkstra run ({dt22:.1f} s)"}
        line["parity_vs_oracle"] = bool((dref == d_host).all())
        bref = oracle_bfs_levels(g, s)
        line["bfs"]["parity_vs_oracle"] = bool((bref == bfs_lv).all())
        line["bfs"]["pull"]["parity_vs_oracle"] = bool((bref == pull_lv).all())
        line["warm_start"]["parity_vs_oracle"] = bool((oracle_sssp_w(g, w2_host, s) == d_warm_host).all())
    if not args.no_functors:
        line["functors"] = bench_functors(llp, dev, cpu=cpu)
    if not args.no_batched:
        line["batched"] = bench_batched(llp, dev, stream, cpu=cpu)
        line["batched_graphs"] = bench_batched_graphs(llp, dev)
    if not args.no_learned:
        line["learned"] = bench_learned(llp, dev, g, s, cpu=cpu, cpu22_s=dt22)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def _ev_time(fn, reps=3, stream=None):
    import torch
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


def smem_peak_gbs(dev):
    """Shared-memory bandwidth of the GPU: 128 B per clock per SM at the maximum SM clock."""
    import torch
    props = torch.cuda.get_device_properties(dev)
    mhz = 2032.0
    try:
        import pynvml
        pynvml.nvmlInit()
        h = pynvml.nvmlDeviceGetHandleByIndex(dev.index if dev.index is not None else 0)
        mhz = float(pynvml.nvmlDeviceGetMaxClockInfo(h, pynvml.NVML_CLOCK_SM))
    except Exception:
        pass
    return props.multi_processor_count * 128.0 * mhz * 1e6 / 1e9, mhz


def batched_oracle(db, knap, job, sm, every_knap=4):
    """The oracle on the batched workload on every host core (instances are independent): every
    job DAG and marriage and every `every_knap`-th knapsack, each checked against the batched
    engine's output; the knapsack time is scaled to the whole family."""
    import functools
    import oracle
    cores, model = cpu_info()
    best = db.t["knap_best"].cpu().numpy()
    comp = db.t["job_completion"].cpu().numpy()
    wife = db.t["sm_wife"].cpu().numpy()
    mo = db.sm_man_off_host
    bad = []

    def k1(i):
        a, b = knap["item_off"][i], knap["item_off"][i + 1]
        if oracle.knapsack(knap["w"][a:b], knap["v"][a:b], int(knap["capacity"][i]))[0] != best[i]:
            bad.append(("knapsack", int(i)))

    def j1(i):
        j0, j1_ = job["job_off"][i], job["job_off"][i + 1]
        off = job["succ_offsets"][j0:j1_ + 1] - job["succ_offsets"][j0]
        ind = job["succ_indices"][job["succ_offsets"][j0]:job["succ_offsets"][j1_]]
        if not (oracle.job_schedule(job["duration"][j0:j1_], off, ind) == comp[j0:j1_]).all():
            bad.append(("job", int(i)))

    def s1(i):
        n = int(sm["n"][i])
        p0 = sm["pref_off"][i]
        r = oracle.stable_marriage(sm["men_pref"][p0:p0 + n * n].reshape(n, n),
                                   sm["women_rank"][p0:p0 + n * n].reshape(n, n))
        if not (r[0] == wife[mo[i]:mo[i + 1]]).all():
            bad.append(("marriage", int(i)))
    kidx = np.arange(0, knap["count"], every_knap)
    t_k = oracle_parallel([functools.partial(k1, i) for i in kidx], cores)
    t_j = oracle_parallel([functools.partial(j1, i) for i in range(job["count"])], cores)
    t_s = oracle_parallel([functools.partial(s1, i) for i in range(sm["count"])], cores)
    t_k_full = t_k * knap["count"] / len(kidx)
    total = t_k_full + t_j + t_s
    count = knap["count"] + job["count"] + sm["count"]
    return {"value": count / total, "unit": "instances/s", "ms": total * 1e3, "cores": cores, "cpu_model": model,
            "kind": "oracle",
            "family_ms": {"knapsack": t_k_full * 1e3, "job": t_j * 1e3, "marriage": t_s * 1e3},
            "sample": f"every job DAG and marriage, every {every_knap}th knapsack (time scaled by "
                      f"{knap['count'] / len(kidx):.2f}); instances spread over {cores} host threads",
            "instances_checked": int(len(kidx) + job["count"] + sm["count"]), "mismatches": bad[:10],
            "parity_vs_oracle": not bad}


def bench_batched(llp, dev, stream, div=1, cpu=True):
    """Batched workload (4,096 knapsack + 2,048 job DAGs + 1,024 stable marriages): one
    persistent launch, autotuned launch shape, replayed from a CUDA graph, against the
    plain engine called once per instance on the same stream (timed on a sample of
    every family and scaled to the full counts).  The knapsack family alone is timed
    too, for its shared-memory roofline.  div > 1 shrinks every family (profiling)."""
    import torch
    import synth
    knap = synth.knapsack_batch(4096 // div)
    job = synth.job_batch(2048 // div)
    sm = synth.marriage_batch(1024 // div)
    db = llp.DeviceBatch(knap, job, sm, device=dev)
    ws = llp.workspace(llp.batch_workspace_size(db), dev)
    cfg, tune_ms, ws = llp.batch_autotune(db, ws=ws, stream=stream)
    st = torch.cuda.Stream(dev)
    with torch.cuda.stream(st):
        llp.batch_solve(db, cfg, ws=ws, stream=st)
    st.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=st):
        llp.batch_solve(db, cfg, ws=ws, stream=st)
    batched_ms = _ev_time(graph.replay, reps=3)
    bst = llp.get_status(ws)
    total = db.count
    cpu_base = batched_oracle(db, knap, job, sm) if cpu else None

    # knapsack family alone: 3 shared-memory accesses of 4 B per cell (two reads of the previous
    # row, one write), Sigma n_i (W_i + 1) cells
    dk = llp.DeviceBatch(knap, None, None, device=dev)
    wsk_b = llp.workspace(llp.batch_workspace_size(dk), dev)
    knap_ms = _ev_time(lambda: llp.batch_solve(dk, cfg, ws=wsk_b, stream=stream), reps=3, stream=stream)
    cells = int(np.sum(np.diff(knap["item_off"]) * (knap["capacity"].astype(np.int64) + 1)))
    peak_smem, sm_mhz = smem_peak_gbs(dev)
    ach = 12.0 * cells / (knap_ms * 1e-3) / 1e9
    knap_roof = {"bound": "smem", "achieved": ach, "peak": peak_smem, "unit": "GB/s", "frac": ach / peak_smem,
                 "cells": cells, "ms": knap_ms, "cells_per_s": cells / (knap_ms * 1e-3),
                 "peak_note": f"SMs x 128 B/clk x {sm_mhz:.0f} MHz (nominal shared-memory bandwidth)",
                 "alg_bytes_per_cell": 12}
    del dk, wsk_b

    # plain engine: one single-instance call per instance (sampled per family)
    wk = torch.from_numpy(knap["w"]).to(dev)
    vk = torch.from_numpy(knap["v"]).to(dev)
    n_max = int(np.diff(knap["item_off"]).max())
    w_max = int(knap["capacity"].max())
    wsk = llp.workspace(llp.lib().llp_knapsack_workspace_size(ctypes.c_int32(n_max), ctypes.c_int32(w_max)), dev)
    best = torch.empty(1, dtype=torch.int32, device=dev)
    kidx = np.arange(0, knap["count"], 16)

    def half_times(run, idx):
        """Times the two interleaved halves of a sample separately; each half's estimate of the
        whole family, their mean, and their relative spread (the sampling error)."""
        est = []
        for part in (idx[0::2], idx[1::2]):
            est.append(_ev_time(lambda: run(part), reps=1) / max(len(part), 1))
        return est

    def plain_knap(idx):
        for i in idx:
            a, b = int(knap["item_off"][i]), int(knap["item_off"][i + 1])
            llp.knapsack(wk[a:b], vk[a:b], int(knap["capacity"][i]), want_row=False, ws=wsk)
    ek = half_times(plain_knap, kidx)
    t_knap = float(np.mean(ek)) * knap["count"]
    jidx = np.arange(0, job["count"], 8)
    jgraphs = []
    for i in jidx:
        j0, j1 = int(job["job_off"][i]), int(job["job_off"][i + 1])
        off = job["succ_offsets"][j0:j1 + 1] - job["succ_offsets"][j0]
        ind = job["succ_indices"][job["succ_offsets"][j0]:job["succ_offsets"][j1]]
        gj = llp.DeviceGraph.from_host(dict(n=j1 - j0, m=len(ind), offsets=off, indices=ind, weights=None), dev)
        jgraphs.append((gj, torch.from_numpy(job["duration"][j0:j1]).to(dev)))
    wsj = llp.workspace(llp.lib().llp_job_schedule_workspace_size(ctypes.c_int32(8192), ctypes.c_int64(0)), dev)

    def plain_job(idx):
        for q in idx:
            gj, dj = jgraphs[q]
            llp.job_schedule(gj, dj, ws=wsj)
    ej = half_times(plain_job, np.arange(len(jgraphs)))
    t_job = float(np.mean(ej)) * job["count"]
    sidx = np.arange(0, sm["count"], 8)
    sins = []
    for i in sidx:
        n = int(sm["n"][i]); p0 = int(sm["pref_off"][i])
        sins.append((torch.from_numpy(sm["men_pref"][p0:p0 + n * n].reshape(n, n)).to(dev),
                     torch.from_numpy(sm["women_rank"][p0:p0 + n * n].reshape(n, n)).to(dev)))
    wss = llp.workspace(llp.lib().llp_stable_marriage_workspace_size(ctypes.c_int32(1024)), dev)

    def plain_sm(idx):
        for q in idx:
            a_, b_ = sins[q]
            llp.stable_marriage(a_, b_, ws=wss, want_husband=False, want_next=False)
    es = half_times(plain_sm, np.arange(len(sins)))
    t_sm = float(np.mean(es)) * sm["count"]
    plain_ms = t_knap + t_job + t_sm
    return {"metric": "instances/s", "instances": total, "batched_ms": batched_ms,
            "batched_inst_per_s": total / (batched_ms * 1e-3), "plain_ms_est": plain_ms,
            "plain_inst_per_s": total / (plain_ms * 1e-3), "speedup": plain_ms / batched_ms,
            "plain_family_ms_est": {"knapsack": t_knap, "job": t_job, "marriage": t_sm},
            "plain_sample": "every 16th knapsack, 8th job DAG and 8th marriage instance, scaled",
            "plain_sampling_rel_err": {f: abs(e[0] - e[1]) / (e[0] + e[1]) for f, e in
                                       (("knapsack", ek), ("job", ej), ("marriage", es))},
            "cfg": {"threads": cfg.threads, "knap_unroll": cfg.knap_unroll, "ctas_per_sm": cfg.ctas_per_sm},
            "autotune": {"candidates": [{"threads": t, "ctas_per_sm": c, "knap_unroll": u, "ms": ms}
                                        for (t, c, u), ms in zip([(t, c, u) for t, c in ((1024, 1), (512, 1), (512, 2),
                                                                                          (256, 2)) for u in (4, 8, 16)],
                                                                 tune_ms)]},
            "autotune_ms": tune_ms,
            "status": bst["status"], "cuda_graph": True, "knapsack_roofline": knap_roof,
            "cpu_baseline": cpu_base}


def bench_batched_graphs(llp, dev):
    """Batched small SSSP/BFS (2,048 graphs of 64-8,192 vertices: uniform, power-law and grid
    instances, every 4th a BFS) in one persistent launch replayed from a CUDA graph, against the
    plain engine called once per graph (every 8th graph timed, scaled)."""
    import torch
    import synth
    gb = synth.graph_batch()
    db = llp.DeviceBatch(graphs=gb, device=dev)
    ws = llp.workspace(llp.batch_workspace_size(db), dev)
    st = torch.cuda.Stream(dev)
    with torch.cuda.stream(st):
        llp.batch_solve(db, ws=ws, stream=st)
    st.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=st):
        llp.batch_solve(db, ws=ws, stream=st)
    batched_ms = _ev_time(graph.replay, reps=5)
    bst = llp.get_status(ws)
    dist_b = db.t["gr_dist"].clone()
    sidx = np.arange(0, gb["count"], 8)
    gs = []
    for i in sidx:
        v0, v1 = int(gb["off"][i]), int(gb["off"][i + 1])
        a, b = int(gb["arc_offsets"][v0]), int(gb["arc_offsets"][v1])
        g = dict(n=v1 - v0, m=b - a, offsets=gb["arc_offsets"][v0:v1 + 1] - a, indices=gb["indices"][a:b],
                 weights=gb["weights"][a:b])
        gs.append((i, llp.DeviceGraph.from_host(g, dev), v0, v1))
    nmax = int(np.diff(gb["off"]).max())
    mmax = max(dg.m for _, dg, _, _ in gs)
    wsp = llp.workspace(llp.sssp_workspace_size(nmax, mmax), dev)
    outp = torch.empty(nmax, dtype=torch.int32, device=dev)

    def plain():
        for i, dg, _, _ in gs:
            f = llp.bfs if gb["unit"][i] else llp.sssp
            f(dg, int(gb["source"][i]), out=outp[:dg.n], ws=wsp)
    plain_ms = _ev_time(plain, reps=1) * gb["count"] / len(sidx)
    same = True
    for i, dg, v0, v1 in gs[:16]:
        f = llp.bfs if gb["unit"][i] else llp.sssp
        f(dg, int(gb["source"][i]), out=outp[:dg.n], ws=wsp)
        same &= bool(torch.equal(outp[:dg.n], dist_b[v0:v1]))
    return {"metric": "instances/s", "instances": gb["count"], "vertices": int(gb["off"][-1]),
            "arcs": int(gb["arc_offsets"][-1]), "batched_ms": batched_ms,
            "batched_inst_per_s": gb["count"] / (batched_ms * 1e-3), "plain_ms_est": plain_ms,
            "plain_inst_per_s": gb["count"] / (plain_ms * 1e-3), "speedup": plain_ms / batched_ms,
            "plain_sample": "every 8th graph through llp_sssp / llp_bfs, scaled",
            "batched_equals_plain_on_16": same, "status": bst["status"], "cuda_graph": True}


def bench_functors(llp, dev, cpu=True):
    """Every other problem of the sweep on its configured workload, device time (CUDA events),
    each beside the oracle on one host core (same instance) and checked against it."""
    import torch
    import synth
    import oracle
    cores, model = cpu_info()

    def cpu_entry(sec, sample="the same instance"):
        return {"ms": sec * 1e3, "cores": 1, "cpu_model": model, "kind": "oracle", "sample": sample}
    out = {}
    # config 1: ER 16,384 / 131,072, source 0 (latency-bound: the input lives in L2)
    g = synth.er16k()
    dg = llp.DeviceGraph.from_host(g, dev)
    ws = llp.workspace(llp.sssp_workspace_size(g["n"], g["m"]), dev)
    d = torch.empty(g["n"], dtype=torch.int32, device=dev)
    t = _ev_time(lambda: llp.sssp(dg, 0, out=d, ws=ws), reps=5)
    st = llp.get_status(ws)
    dres = llp.as_u32(d)
    tb = _ev_time(lambda: llp.bfs(dg, 0, out=d, ws=ws), reps=5)
    bres = llp.as_u32(d)
    out["er16k_sssp"] = {"ms": t, "sweeps": st["sweeps"], "gteps": g["m"] / (t * 1e-3) / 1e9}
    out["er16k_bfs"] = {"ms": tb, "gteps": g["m"] / (tb * 1e-3) / 1e9}
    if cpu:
        tc, ref = cpu_time(lambda: oracle.sssp(g["offsets"], g["indices"], g["weights"], 0))
        out["er16k_sssp"].update(cpu_baseline=cpu_entry(tc), parity_vs_oracle=bool((dres == ref).all()))
        tc, ref = cpu_time(lambda: oracle.bfs(g["offsets"], g["indices"], 0))
        out["er16k_bfs"].update(cpu_baseline=cpu_entry(tc), parity_vs_oracle=bool((bres == ref).all()))
    # config 3: stable marriage, n = 16,384 random and n = 8,192 with one shared men's order
    for name, n, adv, seed in (("marriage16384_random", 16384, False, 3), ("marriage8192_shared", 8192, True, 4)):
        mp, wr = synth.marriage(n, seed=seed, adversarial=adv)
        tmp, twr = torch.from_numpy(mp).to(dev), torch.from_numpy(wr).to(dev)
        wife, _, _, wsm = llp.stable_marriage(tmp, twr)
        t = _ev_time(lambda: llp.stable_marriage(tmp, twr, ws=wsm, want_husband=False, want_next=False), reps=3)
        st = llp.get_status(wsm)
        out[name] = {"ms": t, "proposals": st["aux"], "proposals_per_s": st["aux"] / (t * 1e-3),
                     "matchings_per_s": 1e3 / t, "status": st["status"]}
        if cpu:
            tc, ref = cpu_time(lambda: oracle.stable_marriage(mp, wr))
            out[name].update(cpu_baseline=cpu_entry(tc), parity_vs_oracle=bool((wife.cpu().numpy() == ref[0]).all()),
                             oracle_proposals=ref[3])
        del tmp, twr, mp, wr
        torch.cuda.empty_cache()
    # 0-1 knapsack, one instance n = 2,048, capacity 65,536
    w, v = synth.knapsack(2048, 65536, seed=5, stream=77)
    tw, tv = torch.from_numpy(w).to(dev), torch.from_numpy(v).to(dev)
    best, _, wsk = llp.knapsack(tw, tv, 65536, want_row=False)
    t = _ev_time(lambda: llp.knapsack(tw, tv, 65536, want_row=False, ws=wsk), reps=3)
    out["knapsack_2048x65536"] = {"ms": t, "cells_per_s": 2048 * 65537 / (t * 1e-3)}
    if cpu:
        tc, ref = cpu_time(lambda: oracle.knapsack(w, v, 65536))
        out["knapsack_2048x65536"].update(cpu_baseline=cpu_entry(tc), parity_vs_oracle=int(best.item()) == ref[0])
    # job scheduling, one DAG of 1,048,576 jobs (Poisson(3) forward arcs)
    gj, dur = synth.job_dag(1 << 20, seed=5)
    dgj = llp.DeviceGraph.from_host(gj, dev)
    td = torch.from_numpy(dur).to(dev)
    comp, wsj = llp.job_schedule(dgj, td)
    t = _ev_time(lambda: llp.job_schedule(dgj, td, ws=wsj), reps=3)
    st = llp.get_status(wsj)
    out["job_1M"] = {"ms": t, "jobs": gj["n"], "arcs": gj["m"], "sweeps": st["sweeps"], "status": st["status"]}
    if cpu:
        tc, ref = cpu_time(lambda: oracle.job_schedule(dur, gj["offsets"], gj["indices"]))
        out["job_1M"].update(cpu_baseline=cpu_entry(tc), parity_vs_oracle=bool((comp.cpu().numpy() == ref).all()))
    # transitive closure of a random DAG, n = 8,192, p = 4/n
    gc = synth.random_dag(8192, 4, seed=6)
    dc = llp.DeviceGraph.from_host(gc, dev)
    R, wsc = llp.transitive_closure(dc)
    t = _ev_time(lambda: llp.transitive_closure(dc, ws=wsc), reps=3)
    st = llp.get_status(wsc)
    out["closure_dag8192"] = {"ms": t, "sweeps": st["sweeps"], "pairs": st["advances"], "status": st["status"]}
    if cpu:
        tc, ref = cpu_time(lambda: oracle.transitive_closure(gc["offsets"], gc["indices"]))
        out["closure_dag8192"].update(cpu_baseline=cpu_entry(tc),
                                      parity_vs_oracle=bool((R.cpu().numpy().view(np.uint32) == ref).all()))
    # reduction of 2^28 uint64 (2 GiB, HBM-bound): roofline against the measured copy bandwidth
    x = torch.randint(-(1 << 62), 1 << 62, (1 << 28,), dtype=torch.int64, device=dev)
    sm, wsr = llp.reduce_sum(x)
    t = _ev_time(lambda: llp.reduce_sum(x, ws=wsr), reps=3)
    peak, kind = peaks()
    gbs = (8 << 28) / (t * 1e-3) / 1e9
    out["reduce_2^28_u64"] = {"ms": t, "GB_per_s": gbs, "frac_of_measured_hbm": gbs / peak}
    if cpu:
        xs = x[: 1 << 24].cpu().numpy().view(np.uint64)
        tc, _ = cpu_time(lambda: oracle.reduce_sum(xs))
        xh = x.cpu().numpy().view(np.uint64)
        out["reduce_2^28_u64"].update(
            cpu_baseline=cpu_entry(tc * 16, sample="the first 2^24 values, time scaled by 16"),
            parity_vs_oracle=(int(sm.item()) & 0xFFFFFFFFFFFFFFFF) == oracle.reduce_sum(xh))
        del xh
    del x
    torch.cuda.empty_cache()
    return out


def bench_learned(llp, dev, g22, s22, cpu=True, cpu22_s=None):
    """Mixed stream: R-MAT scale 20/22/24 SSSP, 2048x2048 grid SSSP, closure of a random
    DAG (n=8192, p=4/n).  Three arms on the same device, end-to-end device time of the stream:
    the learned schedule (network on the device), the plain engine's fixed heuristic schedule,
    and the plain engine autotuned per item (coordinate search over mode, bucket width, block
    configuration and local chain, each candidate timed; the search itself is not counted).
    Every item's result is compared with the heuristic run (bit-exact) and, on the host, with
    the oracle (one core; R-MAT 22 reuses the headline's oracle run)."""
    import torch
    import synth
    import oracle
    from paper_2603_13147_b300 import sched as S
    if not os.path.exists(S.MODEL_PATH):
        return {"unavailable": "no trained scheduler model in the package"}
    cores, model = cpu_info()
    params = S.load_model(device=dev)
    items = []
    for scale in (20, 22, 24):
        gg = g22 if scale == 22 else synth.rmat(scale, seed=6 + scale)
        src = s22 if scale == 22 else synth.max_out_degree_vertex(gg)
        items.append((f"rmat{scale}_sssp", gg, src))
    items.append(("grid2048_sssp", synth.grid_graph(2048, 2048, 1, 1000, seed=6), 0))
    res = {}
    tot_h = tot_l = tot_a = tot_cpu = 0.0
    parity_all = True
    for name, gg, src in items:
        dg = llp.DeviceGraph.from_host(gg, dev)
        ws = llp.workspace(llp.sssp_workspace_size(gg["n"], gg["m"]), dev)
        out = torch.empty(gg["n"], dtype=torch.int32, device=dev)
        th = _ev_time(lambda: llp.sssp(dg, src, out=out, ws=ws), reps=3)
        ref = out.clone()
        ls = S.learned_sched(params)
        tl = _ev_time(lambda: llp.sssp(dg, src, out=out, ws=ws, sched=ls), reps=3)
        st = llp.get_status(ws)
        same_l = bool(torch.equal(ref, out))
        wmax = S.sampled_wmax(gg)
        t_search = time.perf_counter()
        label, log, _ = S.label_graph(dg, src, False, wmax, ws=ws)
        t_search = time.perf_counter() - t_search
        asch = S.label_to_sched(label, wmax)
        ta = _ev_time(lambda: llp.sssp(dg, src, out=out, ws=ws, sched=asch), reps=3)
        same_a = bool(torch.equal(ref, out))
        ent = {"heuristic_ms": th, "learned_ms": tl, "autotuned_ms": ta,
               "learned_schedule": [st["mode_used"], st["delta_used"], st["block_cfg_used"],
                                    st["local_chain_used"]],
               "learned_schedule_fields": ["mode", "delta", "block_cfg", "local_chain"],
               "autotuned_schedule": {"mode": int(label[0]), "delta": S.delta_of_class(int(label[1]), wmax),
                                      "block_cfg": int(label[2]) + 1,
                                      "local_chain": S.CHAIN_OF_CLASS[int(label[3])],
                                      "group_words": S.GW_OF_CLASS[int(label[4])]},
               "autotune_candidates": len(log), "autotune_search_s": t_search,
               "bit_exact": same_l and same_a}
        if cpu:
            if name == "rmat22_sssp" and cpu22_s is not None:
                tc = cpu22_s
                ok = None
            else:
                tc, dref = cpu_time(lambda: oracle.sssp(gg["offsets"], gg["indices"], gg["weights"], src))
                ok = bool((llp.as_u32(ref) == dref).all())
                parity_all &= ok
            ent["cpu_baseline_ms"] = tc * 1e3
            ent["parity_vs_oracle"] = ok
            tot_cpu += tc
        res[name] = ent
        tot_h += th
        tot_l += tl
        tot_a += ta
        del dg, ws, out
        torch.cuda.empty_cache()
    gc = synth.random_dag(8192, 4, seed=6)
    dc = llp.DeviceGraph.from_host(gc, dev)
    R, wsc = llp.transitive_closure(dc)
    tc_ms = _ev_time(lambda: llp.transitive_closure(dc, ws=wsc), reps=3)
    res["closure8192"] = {"heuristic_ms": tc_ms, "learned_ms": tc_ms, "autotuned_ms": tc_ms,
                          "note": "no schedule choice"}
    if cpu:
        tcc, Rref = cpu_time(lambda: oracle.transitive_closure(gc["offsets"], gc["indices"]))
        ok = bool((R.cpu().numpy().view(np.uint32) == Rref).all())
        parity_all &= ok
        res["closure8192"].update(cpu_baseline_ms=tcc * 1e3, parity_vs_oracle=ok)
        tot_cpu += tcc
    tot_h += tc_ms
    tot_l += tc_ms
    tot_a += tc_ms
    line = {"stream_heuristic_ms": tot_h, "stream_learned_ms": tot_l, "stream_autotuned_ms": tot_a,
            "speedup_vs_heuristic": tot_h / tot_l, "speedup_vs_autotuned": tot_a / tot_l,
            "items": res}
    if cpu:
        line["cpu_baseline"] = {"ms": tot_cpu * 1e3, "cores": 1, "cpu_model": model, "kind": "oracle",
                                "sample": "every item of the stream on one host core (Dijkstra per SSSP item, "
                                          "Warshall for the closure)"}
        line["parity_vs_oracle"] = parity_all
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="llp", choices=["llp", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-engine section")
    ap.add_argument("--no-functors", action="store_true", help="skip the other-problems section")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-scheduler stream section")
    ap.add_argument("--scale", type=int, default=SCALE, help="R-MAT scale (22 = the benchmarked workload; "
                    "smaller scales are for profiling captures)")
    ap.add_argument("--batched-only", type=int, default=0, metavar="DIV",
                    help="profiling: run only the batched section with every family divided by DIV, "
                         "print its JSON and exit (not a benchmark line)")
    args = ap.parse_args()
    if args.batched_only:
        import torch
        import paper_2603_13147_b300 as llp
        dev = torch.device("cuda", 0)
        llp.lib()
        print(json.dumps(bench_batched(llp, dev, torch.cuda.current_stream(dev), div=args.batched_only)))
        return 0
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
