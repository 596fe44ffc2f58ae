"""The caller-owned workspace (the boundary's ws / ws_bytes): the library
takes every device buffer of a graph from it and allocates nothing."""
import os
import re

import numpy as np
import pytest

from paper_2511_10073_gb300 import netgen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_library_source_allocates_no_device_memory():
    csrc = os.path.join(ROOT, "paper_2511_10073_gb300", "csrc")
    for f in os.listdir(csrc):
        src = open(os.path.join(csrc, f)).read()
        for call in ("cudaMalloc", "cudaFree", "cudaMallocAsync", "cudaMallocManaged",
                     "cudaHostAlloc", "cudaMallocHost"):
            assert not re.search(r"\b%s\s*\(" % call, src), (f, call)


def test_workspace_bound_on_the_host():
    import paper_2511_10073_gb300 as pl
    pl.lib()
    small = netgen.make_netlist("tiny", 1)
    big = netgen.make_netlist("small", 1)
    prm = pl.params(nbx=16, nby=16)
    # built from sizes alone: the arrays are host numpy here, never read
    class Fake:
        def __init__(self, nl):
            s = pl.PlNetlist()
            s.num_cells, s.num_nets, s.num_pins = nl.num_cells, nl.num_nets, nl.num_pins
            s.xl, s.yl, s.xh, s.yh = nl.region
            self.struct = s
    a, b = pl.pl_workspace_size(Fake(small), prm), pl.pl_workspace_size(Fake(big), prm)
    assert 0 < a and 0 < b
    assert pl.pl_workspace_size(Fake(small), pl.params(nbx=16, nby=16, wdtype=2)) <= a
    f = Fake(small)
    f.struct.num_cells = -1
    assert pl.pl_workspace_size(f, prm) == 0


torch = pytest.importorskip("torch")


@pytest.mark.gpu
def test_too_small_workspace_is_reported():
    import paper_2511_10073_gb300 as pl
    nl = netgen.make_netlist("tiny", 2)
    dnl = pl.DeviceNetlist(nl)
    prm = pl.params(nbx=16, nby=16)
    with pytest.raises(pl.PlError) as e:
        pl.pl_build_graph(dnl, prm, ws=pl.workspace(1 << 16))
    assert e.value.code == pl.PL_ERR_WORKSPACE
    assert "workspace too small" in str(e.value)
    with pytest.raises(pl.PlError) as e:
        pl.pl_build_graph(dnl, prm, ws=pl.workspace(1 << 20)[1:])  # not 256-byte aligned
    assert e.value.code == pl.PL_ERR_INVALID_ARG


@pytest.mark.gpu
@pytest.mark.parametrize("cfg,kw", [
    ("micro", dict(nbx=4, nby=4)), ("small", dict(nbx=8, nby=8, det_ratio=0.4)),
    ("tiny", dict(nbx=96, nby=80, wdtype=2)), ("medium", dict(nbx=32, nby=32)),
    ("large", dict(nbx=32, nby=32, wdtype=2, ntaps=3, tap_k=(2, 4, 8, 0),
                   tap_alpha=(1 / 3, 1 / 3, 1 / 3, 0)))])
def test_bound_covers_the_whole_initializer(cfg, kw):
    """pl_workspace_size suffices for the static build, every refinement round
    and the filters; a workspace of exactly the bytes that run used suffices
    again (the requests are a fixed sequence)."""
    import paper_2511_10073_gb300 as pl
    nl = netgen.make_netlist(cfg, 1)
    dnl = pl.DeviceNetlist(nl)
    prm = pl.params(**kw)
    bound = pl.pl_workspace_size(dnl, prm)
    g = pl.pl_build_graph(dnl, prm)
    out = torch.empty(nl.num_cells * 2, dtype=torch.float32, device="cuda")
    pl.pl_filter_init(g, prm, 1, None, out)
    info = g.info()
    assert info["ws_bytes"] == bound and 0 < info["ws_static"] <= info["ws_peak"] <= bound
    peak = info["ws_peak"]
    g.destroy()
    g2 = pl.pl_build_graph(dnl, prm, ws=pl.workspace(peak))
    out2 = torch.empty_like(out)
    pl.pl_filter_init(g2, prm, 1, None, out2)
    torch.cuda.synchronize()
    assert torch.equal(out, out2)
    print(f"{cfg}: bound {bound / 2**20:.1f} MiB, used {peak / 2**20:.1f} MiB")


@pytest.mark.gpu
def test_repeated_steps_allocate_nothing():
    """Build, initializer and HPWL steps after the first leave the device's
    free memory unchanged: no allocation by the library (or the binding)."""
    import paper_2511_10073_gb300 as pl
    nl = netgen.make_netlist("small", 3)
    dnl = pl.DeviceNetlist(nl)
    prm = pl.params(nbx=8, nby=8, det_ratio=0.4)
    g = pl.pl_build_graph(dnl, prm)
    out = torch.empty(nl.num_cells * 2, dtype=torch.float32, device="cuda")
    hws = pl.hpwl_workspace(nl.num_nets)
    h = torch.zeros(1, dtype=torch.float64, device="cuda")

    def step():
        pl.pl_build_graph(dnl, prm, graph=g)
        pl.pl_filter_init(g, prm, 1, None, out)
        pl.pl_hpwl(dnl, out, h, hws)

    step()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    ws0 = g.ws.data_ptr()
    for _ in range(5):
        step()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert g.ws.data_ptr() == ws0
    assert np.isfinite(h.item())
