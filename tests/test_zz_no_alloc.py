"""The SSSP entry point for callers that cannot allocate device memory.

llp_sssp_noalloc takes its scratch from a fixed array inside the library
instead of a caller workspace.  These checks call it through the C ABI and
compare it with llp_sssp bit for bit, twice in a row (the shared scratch keeps
the previous call's contents, so the second call checks that everything that
must start cleared is cleared).  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth


def _llp():
    import paper_2603_13147_b300 as llp
    llp.build()
    return llp


def test_noalloc_rejects_graphs_beyond_its_scratch():
    """Host-side size check: no GPU work is enqueued for a graph that does not fit."""
    llp = _llp()
    cap = llp.sssp_noalloc_max_workspace()
    assert cap == 64 << 20
    c = llp.Csr()
    c.n, c.m, c.offsets_64 = 4_194_304, 67_108_864, 0
    c.offsets, c.indices, c.weights = 0x1000, 0x2000, 0x3000
    assert llp.sssp_workspace_size(c.n, c.m) > cap
    rc = llp.lib().llp_sssp_noalloc(ctypes.byref(c), 0, ctypes.c_void_p(0x4000), None, None)
    assert rc == llp.LLP_ERR_WORKSPACE_TOO_SMALL


@pytest.mark.gpu
@pytest.mark.parametrize("which", ["er16k", "rmat18"])
def test_noalloc_matches_workspace_entry_point_twice(which):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    llp = _llp()
    if which == "er16k":
        g, s = synth.er16k(), 0
    else:
        g = synth.rmat(18, seed=7)
        s = synth.max_out_degree_vertex(g)
    assert llp.sssp_workspace_size(g["n"], g["m"]) <= llp.sssp_noalloc_max_workspace()
    dg = llp.DeviceGraph.from_host(g, "cuda")
    ref, ws = llp.sssp(dg, s)
    assert llp.get_status(ws)["status"] == 0
    ref = llp.as_u32(ref)
    assert (ref == oracle.sssp(g["offsets"], g["indices"], g["weights"], s)).all()
    out = torch.empty(g["n"], dtype=torch.int32, device="cuda")
    for _ in range(2):
        out.fill_(-1)
        llp.sssp_noalloc(dg, s, out=out)
        torch.cuda.synchronize()
        assert (llp.as_u32(out) == ref).all()


@pytest.mark.gpu
def test_noalloc_larger_then_smaller_graph_and_no_allocation():
    """A large graph, then a small one on the same array: the small call's layout
    sits at other offsets over the large call's leftovers, and must still match the
    oracle.  Free device memory is unchanged across the second call."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    llp = _llp()
    gl = synth.rmat(18, seed=7)
    sl = synth.max_out_degree_vertex(gl)
    gs = synth.er16k()
    dl = llp.DeviceGraph.from_host(gl, "cuda")
    ds = llp.DeviceGraph.from_host(gs, "cuda")
    outl = torch.empty(gl["n"], dtype=torch.int32, device="cuda")
    outs = torch.empty(gs["n"], dtype=torch.int32, device="cuda")
    llp.sssp_noalloc(dl, sl, out=outl)
    assert llp.sssp_noalloc_status() == 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    llp.sssp_noalloc(ds, 0, out=outs)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert llp.sssp_noalloc_status() == 0
    assert (llp.as_u32(outl) == oracle.sssp(gl["offsets"], gl["indices"], gl["weights"], sl)).all()
    assert (llp.as_u32(outs) == oracle.sssp(gs["offsets"], gs["indices"], gs["weights"], 0)).all()


@pytest.mark.gpu
def test_noalloc_status_reports_device_timeout():
    """The device-side outcome is readable: a 1 ns deadline makes the first bounded
    wait give up (LLP_ERR_TIMEOUT); the next call with the default deadline is clean
    and correct."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    llp = _llp()
    g = synth.er16k()
    dg = llp.DeviceGraph.from_host(g, "cuda")
    out = torch.empty(g["n"], dtype=torch.int32, device="cuda")
    llp.sssp_noalloc(dg, 0, out=out, sched=llp.make_sched(deadline_ns=1))
    assert llp.sssp_noalloc_status() == llp.LLP_ERR_TIMEOUT
    llp.sssp_noalloc(dg, 0, out=out)
    assert llp.sssp_noalloc_status() == 0
    assert (llp.as_u32(out) == oracle.sssp(g["offsets"], g["indices"], g["weights"], 0)).all()
