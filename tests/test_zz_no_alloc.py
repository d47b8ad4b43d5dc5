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
