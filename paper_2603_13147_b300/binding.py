"""Thin ctypes binding over libllp.so (include/llp.h).

Argument marshalling only: torch tensors supply device memory and streams, every
step of every sweep runs in the library's CUDA kernels.  There is no CPU
fallback: if libllp.so is missing or no CUDA device is present the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libllp.so")

LLP_OK = 0
LLP_ERR_INVALID_ARG = 1
LLP_ERR_WORKSPACE_TOO_SMALL = 2
LLP_ERR_CUDA = 3
LLP_ERR_TIMEOUT = 4
LLP_ERR_INFEASIBLE = 5
LLP_ERR_OVERFLOW = 6
LLP_ERR_UNSUPPORTED = 7

MODE_AUTO, MODE_SPARSE, MODE_DENSE = 0, 1, 2
DELTA_INF = 0xFFFFFFFF
INF = 0xFFFFFFFF


class LlpError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {status_string(code)} ({code})")
        self.code = code


class Csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("offsets_64", ctypes.c_int32), ("m", ctypes.c_int64),
                ("offsets", ctypes.c_void_p), ("indices", ctypes.c_void_p), ("weights", ctypes.c_void_p)]


class Sched(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("delta", ctypes.c_uint32), ("block_cfg", ctypes.c_int32),
                ("dense_permille", ctypes.c_int32), ("use_mlp", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("deadline_ns", ctypes.c_int64), ("mlp_params", ctypes.c_void_p), ("local_chain", ctypes.c_int32),
                ("pull_permille", ctypes.c_int32), ("group_words", ctypes.c_int32),
                ("fixed_memo", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("sweeps", ctypes.c_int32), ("items", ctypes.c_int64),
                ("edges", ctypes.c_int64), ("advances", ctypes.c_int64), ("aux", ctypes.c_int64),
                ("elapsed_ns", ctypes.c_int64), ("mode_used", ctypes.c_int32), ("delta_used", ctypes.c_uint32),
                ("block_cfg_used", ctypes.c_int32), ("dense_sweeps", ctypes.c_int32),
                ("local_chain_used", ctypes.c_int32), ("pull_sweeps", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib() -> ctypes.CDLL:
    """Load libllp.so; raises if it is missing (no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libllp.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        L.llp_version.restype = ctypes.c_char_p
        L.llp_status_string.restype = ctypes.c_char_p
        for name in ("llp_sssp_workspace_size", "llp_bfs_workspace_size", "llp_stable_marriage_workspace_size",
                     "llp_knapsack_workspace_size", "llp_transitive_closure_workspace_size",
                     "llp_job_schedule_workspace_size", "llp_reduce_workspace_size",
                     "llp_csr_transpose_workspace_size"):
            if hasattr(L, name):
                getattr(L, name).restype = ctypes.c_size_t
        _lib = L
    return _lib


def version() -> str:
    return lib().llp_version().decode()


def status_string(code: int) -> str:
    return lib().llp_status_string(ctypes.c_int32(code)).decode()


def make_sched(mode=0, delta=0, block_cfg=0, dense_permille=0, use_mlp=0, threads=0, deadline_ns=0,
               mlp_params=None, local_chain=0, pull_permille=0, group_words=0, fixed_memo=0) -> Sched:
    s = Sched()
    s.group_words = group_words
    s.fixed_memo = fixed_memo
    s.local_chain = local_chain
    s.pull_permille = pull_permille
    s.mode, s.delta, s.block_cfg, s.dense_permille = mode, delta, block_cfg, dense_permille
    s.use_mlp, s.threads, s.deadline_ns = use_mlp, threads, deadline_ns
    s.mlp_params = None if mlp_params is None else mlp_params.data_ptr()
    return s


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check(rc, what):
    if rc != LLP_OK:
        raise LlpError(rc, what)


def _dev(t, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def workspace(nbytes: int, device=None) -> torch.Tensor:
    """Device workspace (uint8, 256-byte aligned by the CUDA caching allocator)."""
    return torch.empty(max(int(nbytes), 4096), dtype=torch.uint8, device=device or "cuda")


def get_status(ws: torch.Tensor, stream=None) -> dict:
    st = Stats()
    rc = lib().llp_get_status(_ptr(ws), _stream(stream), ctypes.byref(st))
    if rc == LLP_ERR_CUDA:
        raise LlpError(rc, "llp_get_status")
    return st.as_dict()


# ------------------------------------------------------------------ graphs

class DeviceGraph:
    """A CSR graph resident on the device (out-arcs)."""

    def __init__(self, offsets: torch.Tensor, indices: torch.Tensor, weights: torch.Tensor | None):
        if offsets.dtype not in (torch.int32, torch.int64):
            raise TypeError("offsets must be int32 or int64")
        _dev(offsets, offsets.dtype, "offsets")
        _dev(indices, torch.int32, "indices")
        if weights is not None:
            _dev(weights, torch.int32 if weights.dtype == torch.int32 else torch.uint32, "weights")
        self.offsets, self.indices, self.weights = offsets, indices, weights
        self.n = offsets.shape[0] - 1
        self.m = indices.shape[0]

    @classmethod
    def from_host(cls, g: dict, device="cuda", offsets_64: bool = False):
        import numpy as np
        off = g["offsets"].astype(np.int64 if offsets_64 else np.int32)
        w = g.get("weights")
        return cls(torch.from_numpy(off).to(device), torch.from_numpy(g["indices"]).to(device),
                   None if w is None else torch.from_numpy(w.view(np.int32)).to(device))

    def csr(self) -> Csr:
        c = Csr()
        c.n, c.m = self.n, self.m
        c.offsets_64 = 1 if self.offsets.dtype == torch.int64 else 0
        c.offsets, c.indices = self.offsets.data_ptr(), self.indices.data_ptr()
        c.weights = None if self.weights is None else self.weights.data_ptr()
        return c

    def transpose(self, with_weights: bool = False, ws=None, stream=None) -> "DeviceGraph":
        """The in-arc CSR (llp_csr_transpose): row v lists the sources of the arcs into v,
        in an unspecified order; same offset type."""
        dev = self.indices.device
        off = torch.empty(self.n + 1, dtype=self.offsets.dtype, device=dev)
        idx = torch.empty(self.m, dtype=torch.int32, device=dev)
        w = None
        if with_weights:
            if self.weights is None:
                raise ValueError("graph has no weights")
            w = torch.empty(self.m, dtype=self.weights.dtype, device=dev)
        if ws is None:
            ws = workspace(lib().llp_csr_transpose_workspace_size(ctypes.c_int32(self.n), ctypes.c_int64(self.m)),
                           dev)
        c = self.csr()
        rc = lib().llp_csr_transpose(ctypes.byref(c), _ptr(off), _ptr(idx), _ptr(w), _ptr(ws),
                                     ctypes.c_size_t(ws.numel()), _stream(stream))
        _check(rc, "llp_csr_transpose")
        t = DeviceGraph(off, idx, w)
        t.transpose_ws = ws
        return t


def sssp_workspace_size(n: int, m: int) -> int:
    return int(lib().llp_sssp_workspace_size(ctypes.c_int32(n), ctypes.c_int64(m)))


def bfs_workspace_size(n: int, m: int) -> int:
    return int(lib().llp_bfs_workspace_size(ctypes.c_int32(n), ctypes.c_int64(m)))


def _graph_call(fn, wsfn, g: DeviceGraph, source, out, sched, ws, stream, what):
    if out is None:
        out = torch.empty(g.n, dtype=torch.int32, device=g.indices.device)
    _dev(out, torch.int32, "out")
    if ws is None:
        ws = workspace(wsfn(g.n, g.m), g.indices.device)
    c = g.csr()
    rc = fn(ctypes.byref(c), ctypes.c_int32(source), _ptr(out), None if sched is None else ctypes.byref(sched),
            _ptr(ws), ctypes.c_size_t(ws.numel()), _stream(stream))
    _check(rc, what)
    return out, ws


def sssp(g: DeviceGraph, source: int, out=None, sched: Sched | None = None, ws=None, stream=None):
    """Shortest-path distances as int32 bit patterns of uint32 (0xFFFFFFFF = unreachable).
    Returns (dist, workspace)."""
    if g.weights is None:
        raise ValueError("sssp needs weights")
    return _graph_call(lib().llp_sssp, sssp_workspace_size, g, source, out, sched, ws, stream, "llp_sssp")


def bfs(g: DeviceGraph, source: int, out=None, sched: Sched | None = None, ws=None, stream=None):
    """BFS levels (uint32 bit patterns in int32; 0xFFFFFFFF = unreachable).  Returns (level, workspace)."""
    return _graph_call(lib().llp_bfs, bfs_workspace_size, g, source, out, sched, ws, stream, "llp_bfs")


def sssp_host_workspace_size(n: int, m: int, offsets_64: bool = False) -> int:
    L = lib()
    L.llp_sssp_host_workspace_size.restype = ctypes.c_size_t
    return int(L.llp_sssp_host_workspace_size(ctypes.c_int32(n), ctypes.c_int64(m),
                                              ctypes.c_int32(1 if offsets_64 else 0)))


def sssp_host(offsets: torch.Tensor, indices: torch.Tensor, weights: torch.Tensor, source: int,
              out: torch.Tensor, sched: Sched | None = None, ws=None, stream=None):
    """llp_sssp_host: the graph and `out` are HOST tensors (pin them for full copy bandwidth);
    copies, sweep and the copy back are enqueued on `stream`; `out` is valid after it is
    synchronised.  Returns (out, workspace)."""
    for t, name in ((offsets, "offsets"), (indices, "indices"), (weights, "weights"), (out, "out")):
        if t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous host tensor")
    if offsets.dtype not in (torch.int32, torch.int64) or indices.dtype != torch.int32 or out.dtype != torch.int32:
        raise TypeError("offsets int32/int64, indices and out int32")
    c = Csr()
    c.n, c.m = offsets.shape[0] - 1, indices.shape[0]
    c.offsets_64 = 1 if offsets.dtype == torch.int64 else 0
    c.offsets, c.indices, c.weights = offsets.data_ptr(), indices.data_ptr(), weights.data_ptr()
    if ws is None:
        ws = workspace(sssp_host_workspace_size(c.n, c.m, bool(c.offsets_64)))
    rc = lib().llp_sssp_host(ctypes.byref(c), ctypes.c_int32(source), _ptr(out),
                             None if sched is None else ctypes.byref(sched), _ptr(ws), ctypes.c_size_t(ws.numel()),
                             _stream(stream))
    _check(rc, "llp_sssp_host")
    return out, ws


def _warm_call(fn, wsfn, g: DeviceGraph, source, dist, seeds, sched, ws, stream, what):
    _dev(dist, torch.int32, "dist")
    if seeds is not None and seeds.numel() > 0:
        _dev(seeds, torch.int32, "seeds")
    n_seeds = 0 if seeds is None else int(seeds.numel())
    if ws is None:
        ws = workspace(wsfn(g.n, g.m), g.indices.device)
    c = g.csr()
    rc = fn(ctypes.byref(c), ctypes.c_int32(source), _ptr(dist), _ptr(seeds) if n_seeds else None,
            ctypes.c_int32(n_seeds), None if sched is None else ctypes.byref(sched), _ptr(ws),
            ctypes.c_size_t(ws.numel()), _stream(stream))
    _check(rc, what)
    return dist, ws


def sssp_warm(g: DeviceGraph, source: int, dist: torch.Tensor, seeds: torch.Tensor | None, sched=None, ws=None,
              stream=None):
    """Incremental SSSP (llp_sssp_warm): `dist` (in/out) holds upper bounds, e.g. the result on the
    graph before weight decreases / arc insertions; `seeds` (int32) the tails of the changed arcs."""
    if g.weights is None:
        raise ValueError("sssp needs weights")
    return _warm_call(lib().llp_sssp_warm, sssp_workspace_size, g, source, dist, seeds, sched, ws, stream,
                      "llp_sssp_warm")


def bfs_warm(g: DeviceGraph, source: int, level: torch.Tensor, seeds: torch.Tensor | None, sched=None, ws=None,
             stream=None):
    """Incremental BFS after arc insertions (llp_bfs_warm)."""
    return _warm_call(lib().llp_bfs_warm, bfs_workspace_size, g, source, level, seeds, sched, ws, stream,
                      "llp_bfs_warm")


def bfs_pull(g: DeviceGraph, g_in: DeviceGraph, source: int, out=None, sched: Sched | None = None, ws=None,
             stream=None):
    """BFS with direction switching (llp_bfs_pull); g_in = g.transpose().  Returns (level, workspace)."""
    if out is None:
        out = torch.empty(g.n, dtype=torch.int32, device=g.indices.device)
    _dev(out, torch.int32, "out")
    if ws is None:
        ws = workspace(bfs_workspace_size(g.n, g.m), g.indices.device)
    c, ci = g.csr(), g_in.csr()
    rc = lib().llp_bfs_pull(ctypes.byref(c), ctypes.byref(ci), ctypes.c_int32(source), _ptr(out),
                            None if sched is None else ctypes.byref(sched), _ptr(ws), ctypes.c_size_t(ws.numel()),
                            _stream(stream))
    _check(rc, "llp_bfs_pull")
    return out, ws


def as_u32(t: torch.Tensor):
    """View an int32 tensor holding uint32 bit patterns as a numpy uint32 array (host)."""
    return t.cpu().numpy().view("uint32")


# ------------------------------------------------------- other LLP problems

def _size(fn, *args):
    return int(fn(*args))


def stable_marriage(men_pref: torch.Tensor, women_rank: torch.Tensor, sched=None, ws=None, stream=None,
                    want_husband=True, want_next=True):
    """Man-optimal stable matching.  men_pref/women_rank: int32 [n, n] on the device.
    Returns (wife, husband|None, next|None, workspace)."""
    _dev(men_pref, torch.int32, "men_pref"); _dev(women_rank, torch.int32, "women_rank")
    n = men_pref.shape[0]
    dev = men_pref.device
    wife = torch.empty(n, dtype=torch.int32, device=dev)
    hus = torch.empty(n, dtype=torch.int32, device=dev) if want_husband else None
    nxt = torch.empty(n, dtype=torch.int32, device=dev) if want_next else None
    L = lib()
    if ws is None:
        ws = workspace(_size(L.llp_stable_marriage_workspace_size, ctypes.c_int32(n)), dev)
    rc = L.llp_stable_marriage(ctypes.c_int32(n), _ptr(men_pref), _ptr(women_rank), _ptr(wife), _ptr(hus),
                               _ptr(nxt), None if sched is None else ctypes.byref(sched), _ptr(ws),
                               ctypes.c_size_t(ws.numel()), _stream(stream))
    _check(rc, "llp_stable_marriage")
    return wife, hus, nxt, ws


def knapsack(w: torch.Tensor, v: torch.Tensor, capacity: int, want_row=True, sched=None, ws=None, stream=None):
    """0-1 knapsack optimum.  Returns (best int32[1], final_row int32[capacity+1] | None, workspace)."""
    _dev(w, torch.int32, "w"); _dev(v, torch.int32, "v")
    dev = w.device
    best = torch.empty(1, dtype=torch.int32, device=dev)
    row = torch.empty(capacity + 1, dtype=torch.int32, device=dev) if want_row else None
    L = lib()
    if ws is None:
        ws = workspace(_size(L.llp_knapsack_workspace_size, ctypes.c_int32(w.shape[0]), ctypes.c_int32(capacity)),
                       dev)
    rc = L.llp_knapsack(ctypes.c_int32(w.shape[0]), _ptr(w), _ptr(v), ctypes.c_int32(capacity), _ptr(best),
                        _ptr(row), None if sched is None else ctypes.byref(sched), _ptr(ws),
                        ctypes.c_size_t(ws.numel()), _stream(stream))
    _check(rc, "llp_knapsack")
    return best, row, ws


def transitive_closure(g: DeviceGraph, sched=None, ws=None, stream=None):
    """Bit-packed reachability: int32 tensor [n, ceil(n/32)] of uint32 bit patterns."""
    W = (g.n + 31) // 32
    reach = torch.empty((g.n, W), dtype=torch.int32, device=g.indices.device)
    L = lib()
    if ws is None:
        ws = workspace(_size(L.llp_transitive_closure_workspace_size, ctypes.c_int32(g.n), ctypes.c_int64(g.m)),
                       g.indices.device)
    c = g.csr()
    rc = L.llp_transitive_closure(ctypes.byref(c), _ptr(reach), None if sched is None else ctypes.byref(sched),
                                  _ptr(ws), ctypes.c_size_t(ws.numel()), _stream(stream))
    _check(rc, "llp_transitive_closure")
    return reach, ws


def job_schedule(succ: DeviceGraph, duration: torch.Tensor, sched=None, ws=None, stream=None):
    """Earliest completion times (int32[n]) of a job DAG given by successor arcs."""
    _dev(duration, torch.int32, "duration")
    comp = torch.empty(succ.n, dtype=torch.int32, device=duration.device)
    L = lib()
    if ws is None:
        ws = workspace(_size(L.llp_job_schedule_workspace_size, ctypes.c_int32(succ.n), ctypes.c_int64(succ.m)),
                       duration.device)
    c = succ.csr()
    rc = L.llp_job_schedule(ctypes.byref(c), _ptr(duration), _ptr(comp), None if sched is None else ctypes.byref(sched),
                            _ptr(ws), ctypes.c_size_t(ws.numel()), _stream(stream))
    _check(rc, "llp_job_schedule")
    return comp, ws


def reduce_sum(x: torch.Tensor, sched=None, ws=None, stream=None):
    """Sum modulo 2^64 of a uint64 vector (given as int64 bit patterns).  Returns (sum int64[1], ws)."""
    _dev(x, torch.int64, "x")
    out = torch.empty(1, dtype=torch.int64, device=x.device)
    L = lib()
    if ws is None:
        ws = workspace(_size(L.llp_reduce_workspace_size, ctypes.c_int64(x.numel())), x.device)
    rc = L.llp_reduce(ctypes.c_int64(x.numel()), _ptr(x), _ptr(out), None if sched is None else ctypes.byref(sched),
                      _ptr(ws), ctypes.c_size_t(ws.numel()), _stream(stream))
    _check(rc, "llp_reduce")
    return out, ws


def sweep_log(ws: torch.Tensor, stream=None, max_records: int = 4096):
    """Per-sweep records of the last SSSP/BFS call on `ws`: numpy uint32 [k, 4]
    (device ns since start, small worklist size, chunk worklist size, flags)."""
    import numpy as np
    buf = np.zeros((max_records, 4), np.uint32)
    cnt = lib().llp_sweep_log(_ptr(ws), _stream(stream), buf.ctypes.data_as(ctypes.c_void_p),
                              ctypes.c_int32(max_records))
    if cnt < 0:
        raise LlpError(-cnt, "llp_sweep_log")
    return buf[:cnt]


def gather_floor(g: DeviceGraph, state: torch.Tensor, sink: torch.Tensor | None = None, stream=None):
    """The access-pattern floor of a push sweep: one pass over every arc of g that streams the CSR
    and reads state[target] at random (llp_gather_floor).  Returns the sink tensor (reuse it)."""
    L = lib()
    L.llp_gather_floor_sink_size.restype = ctypes.c_size_t
    nbytes = int(L.llp_gather_floor_sink_size())
    if sink is None:
        sink = torch.empty(nbytes, dtype=torch.uint8, device=g.indices.device)
    _dev(state, torch.int32, "state")
    c = g.csr()
    rc = L.llp_gather_floor(ctypes.byref(c), _ptr(state), _ptr(sink), ctypes.c_size_t(sink.numel()), _stream(stream))
    _check(rc, "llp_gather_floor")
    return sink


def sssp_noalloc_max_workspace() -> int:
    L = lib()
    L.llp_sssp_noalloc_max_workspace.restype = ctypes.c_size_t
    return int(L.llp_sssp_noalloc_max_workspace())


def sssp_noalloc(g: DeviceGraph, source: int, out=None, sched: Sched | None = None, stream=None):
    """SSSP without a caller workspace (the library's fixed 64 MiB scratch array).

    For callers that cannot allocate device memory themselves.  `out` must be
    given by such callers; when it is None this wrapper creates it with torch,
    which is for convenience in Python only.  Calls on one device must not
    overlap on the GPU; the first call on a device must precede any stream
    capture.  Returns dist (uint32 bit patterns in int32)."""
    if g.weights is None:
        raise ValueError("sssp needs weights")
    if out is None:
        out = torch.empty(g.n, dtype=torch.int32, device=g.indices.device)
    _dev(out, torch.int32, "out")
    c = g.csr()
    rc = lib().llp_sssp_noalloc(ctypes.byref(c), ctypes.c_int32(source), _ptr(out),
                                None if sched is None else ctypes.byref(sched), _stream(stream))
    _check(rc, "llp_sssp_noalloc")
    return out


def sssp_noalloc_status(stream=None) -> int:
    """Device status of the last llp_sssp_noalloc call on the current device
    (0 = LLP_OK); synchronises the stream."""
    st = ctypes.c_int32(0)
    rc = lib().llp_sssp_noalloc_status(ctypes.byref(st), _stream(stream))
    _check(rc, "llp_sssp_noalloc_status")
    return int(st.value)


# ------------------------------------------------------------------ batched

class Batch(ctypes.Structure):
    _fields_ = [("knap_count", ctypes.c_int32), ("knap_max_capacity", ctypes.c_int32),
                ("knap_item_off", ctypes.c_void_p), ("knap_w", ctypes.c_void_p), ("knap_v", ctypes.c_void_p),
                ("knap_capacity", ctypes.c_void_p), ("knap_best", ctypes.c_void_p),
                ("job_count", ctypes.c_int32), ("job_max_n", ctypes.c_int32),
                ("job_off", ctypes.c_void_p), ("job_succ_offsets", ctypes.c_void_p),
                ("job_succ_indices", ctypes.c_void_p), ("job_duration", ctypes.c_void_p),
                ("job_completion", ctypes.c_void_p),
                ("sm_count", ctypes.c_int32), ("sm_max_n", ctypes.c_int32),
                ("sm_n", ctypes.c_void_p), ("sm_pref_off", ctypes.c_void_p), ("sm_man_off", ctypes.c_void_p),
                ("sm_men_pref", ctypes.c_void_p), ("sm_women_rank", ctypes.c_void_p), ("sm_wife", ctypes.c_void_p),
                ("gr_count", ctypes.c_int32), ("gr_max_n", ctypes.c_int32),
                ("gr_off", ctypes.c_void_p), ("gr_arc_offsets", ctypes.c_void_p), ("gr_indices", ctypes.c_void_p),
                ("gr_weights", ctypes.c_void_p), ("gr_source", ctypes.c_void_p), ("gr_unit", ctypes.c_void_p),
                ("gr_dist", ctypes.c_void_p)]


class BatchCfg(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("knap_unroll", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class DeviceBatch:
    """Device-resident batch of knapsack / job-DAG / stable-marriage / small SSSP-BFS instances
    (host dicts as produced by synth.knapsack_batch / job_batch / marriage_batch / graph_batch)."""

    def __init__(self, knap=None, job=None, sm=None, graphs=None, device="cuda"):
        import numpy as np
        d = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).to(device)
        self.device = device
        self.t = {}
        self.knap_count = self.job_count = self.sm_count = self.gr_count = 0
        self.knap_max_capacity = self.job_max_n = self.sm_max_n = self.gr_max_n = 0
        if knap is not None and knap["count"] > 0:
            self.knap_count = int(knap["count"])
            self.knap_max_capacity = int(knap["capacity"].max())
            self.t.update(knap_item_off=d(knap["item_off"], np.int64), knap_w=d(knap["w"], np.int32),
                          knap_v=d(knap["v"], np.int32), knap_capacity=d(knap["capacity"], np.int32),
                          knap_best=torch.empty(self.knap_count, dtype=torch.int32, device=device))
        if job is not None and job["count"] > 0:
            self.job_count = int(job["count"])
            self.job_max_n = int(np.diff(job["job_off"]).max())
            self.t.update(job_off=d(job["job_off"], np.int64), job_succ_offsets=d(job["succ_offsets"], np.int64),
                          job_succ_indices=d(job["succ_indices"], np.int32),
                          job_duration=d(job["duration"], np.int32),
                          job_completion=torch.empty(int(job["job_off"][-1]), dtype=torch.int32, device=device))
        if sm is not None and sm["count"] > 0:
            self.sm_count = int(sm["count"])
            self.sm_max_n = int(sm["n"].max())
            man_off = np.zeros(self.sm_count + 1, np.int64)
            man_off[1:] = np.cumsum(sm["n"])
            self.sm_man_off_host = man_off
            self.t.update(sm_n=d(sm["n"], np.int32), sm_pref_off=d(sm["pref_off"], np.int64),
                          sm_man_off=d(man_off, np.int64), sm_men_pref=d(sm["men_pref"], np.int32),
                          sm_women_rank=d(sm["women_rank"], np.int32),
                          sm_wife=torch.empty(int(man_off[-1]), dtype=torch.int32, device=device))
        if graphs is not None and graphs["count"] > 0:
            self.gr_count = int(graphs["count"])
            self.gr_max_n = int(np.diff(graphs["off"]).max())
            self.t.update(gr_off=d(graphs["off"], np.int64), gr_arc_offsets=d(graphs["arc_offsets"], np.int64),
                          gr_indices=d(graphs["indices"], np.int32), gr_source=d(graphs["source"], np.int32),
                          gr_dist=torch.empty(int(graphs["off"][-1]), dtype=torch.int32, device=device))
            if graphs.get("weights") is not None:
                self.t["gr_weights"] = d(np.asarray(graphs["weights"]).view(np.int32), np.int32)
            if graphs.get("unit") is not None:
                self.t["gr_unit"] = d(graphs["unit"], np.int32)

    def struct(self) -> Batch:
        b = Batch()
        b.knap_count, b.knap_max_capacity = self.knap_count, self.knap_max_capacity
        b.job_count, b.job_max_n = self.job_count, self.job_max_n
        b.sm_count, b.sm_max_n = self.sm_count, self.sm_max_n
        b.gr_count, b.gr_max_n = self.gr_count, self.gr_max_n
        for k, v in self.t.items():
            setattr(b, k, v.data_ptr())
        return b

    @property
    def count(self):
        return self.knap_count + self.job_count + self.sm_count + self.gr_count


def batch_workspace_size(db: DeviceBatch) -> int:
    L = lib()
    L.llp_batch_workspace_size.restype = ctypes.c_size_t
    b = db.struct()
    return int(L.llp_batch_workspace_size(ctypes.byref(b)))


def batch_solve(db: DeviceBatch, cfg: BatchCfg | None = None, sched=None, ws=None, stream=None):
    """Solves every instance of the batch in one persistent launch.  Returns the workspace."""
    if ws is None:
        ws = workspace(batch_workspace_size(db), db.device)
    b = db.struct()
    rc = lib().llp_batch_solve(ctypes.byref(b), None if cfg is None else ctypes.byref(cfg),
                               None if sched is None else ctypes.byref(sched), _ptr(ws), ctypes.c_size_t(ws.numel()),
                               _stream(stream))
    _check(rc, "llp_batch_solve")
    return ws


def batch_autotune(db: DeviceBatch, ws=None, stream=None):
    """Times every candidate launch shape; returns (best BatchCfg, list of ms, workspace)."""
    if ws is None:
        ws = workspace(batch_workspace_size(db), db.device)
    b = db.struct()
    best = BatchCfg()
    ms = (ctypes.c_float * 16)()
    n = ctypes.c_int32(0)
    rc = lib().llp_batch_autotune(ctypes.byref(b), _ptr(ws), ctypes.c_size_t(ws.numel()), _stream(stream),
                                  ctypes.byref(best), ms, ctypes.c_int32(16), ctypes.byref(n))
    _check(rc, "llp_batch_autotune")
    return best, [float(ms[i]) for i in range(n.value)], ws


# -------------------------------------------------------- learned scheduler

class MlpDims(ctypes.Structure):
    _fields_ = [("F", ctypes.c_int32), ("H1", ctypes.c_int32), ("H2", ctypes.c_int32), ("O", ctypes.c_int32),
                ("nheads", ctypes.c_int32), ("heads", ctypes.c_int32 * 8)]


SCHED_F, SCHED_H1, SCHED_H2 = 16, 64, 64
SCHED_HEADS = (3, 8, 3, 4, 5)  # mode, bucket-width class, block_cfg, local-chain class, group-width class


def mlp_dims(F=SCHED_F, H1=SCHED_H1, H2=SCHED_H2, heads=SCHED_HEADS) -> MlpDims:
    d = MlpDims()
    d.F, d.H1, d.H2, d.O, d.nheads = F, H1, H2, sum(heads), len(heads)
    for i, h in enumerate(heads):
        d.heads[i] = h
    return d


def mlp_param_count(d: MlpDims) -> int:
    L = lib()
    L.llp_mlp_param_count.restype = ctypes.c_size_t
    return int(L.llp_mlp_param_count(ctypes.byref(d)))


def mlp_forward(d: MlpDims, params: torch.Tensor, X: torch.Tensor, stream=None) -> torch.Tensor:
    _dev(params, torch.float32, "params"); _dev(X, torch.float32, "X")
    out = torch.empty((X.shape[0], d.O), dtype=torch.float32, device=X.device)
    rc = lib().llp_mlp_forward(ctypes.byref(d), _ptr(params), _ptr(X), ctypes.c_int32(X.shape[0]), _ptr(out),
                               _stream(stream))
    _check(rc, "llp_mlp_forward")
    return out


def mlp_loss_grad(d: MlpDims, params: torch.Tensor, X: torch.Tensor, Y: torch.Tensor, ws=None, stream=None):
    """Returns (loss tensor[1], grad tensor like params, workspace)."""
    _dev(params, torch.float32, "params"); _dev(X, torch.float32, "X"); _dev(Y, torch.int32, "Y")
    L = lib()
    L.llp_mlp_workspace_size.restype = ctypes.c_size_t
    B = X.shape[0]
    if ws is None:
        ws = workspace(L.llp_mlp_workspace_size(ctypes.byref(d), ctypes.c_int32(B)), X.device)
    loss = torch.empty(1, dtype=torch.float32, device=X.device)
    grad = torch.empty_like(params)
    rc = L.llp_mlp_loss_grad(ctypes.byref(d), _ptr(params), _ptr(X), _ptr(Y), ctypes.c_int32(B), _ptr(loss),
                             _ptr(grad), _ptr(ws), ctypes.c_size_t(ws.numel()), _stream(stream))
    _check(rc, "llp_mlp_loss_grad")
    return loss, grad, ws


def mlp_adam(params, grad, m, v, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    rc = lib().llp_mlp_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), ctypes.c_size_t(params.numel()),
                            ctypes.c_int32(step), ctypes.c_float(lr), ctypes.c_float(beta1), ctypes.c_float(beta2),
                            ctypes.c_float(eps), _stream(stream))
    _check(rc, "llp_mlp_adam")


def graph_schedule(g: DeviceGraph, source: int, params: torch.Tensor, unit_weights=False, ws=None, stream=None):
    """Runs the device feature + inference kernels; returns (chosen Sched, features list)."""
    if ws is None:
        ws = workspace(1 << 16, g.indices.device)
    chosen = Sched()
    feats = (ctypes.c_float * 16)()
    c = g.csr()
    rc = lib().llp_graph_schedule(ctypes.byref(c), ctypes.c_int32(source), ctypes.c_int32(1 if unit_weights else 0),
                                  _ptr(params), _ptr(ws), ctypes.c_size_t(ws.numel()), _stream(stream),
                                  ctypes.byref(chosen), feats)
    _check(rc, "llp_graph_schedule")
    return chosen, [float(x) for x in feats]
