"""The allocation-free HPWL entry point (pl_hpwl_noalloc).

Some callers cannot allocate device memory or hand scratch memory to a
library: a host framework that owns every device allocation through its own
pool and gives plug-ins no allocator, or a code path where an allocation
(which may synchronize the device) is not allowed.  pl_hpwl_noalloc serves
them with a fixed scratch array inside the library.  These tests call it
through the C ABI and check it against pl_hpwl (same kernel and grid, so the
same bits) and against the FP64 oracle's HPWL, on two calls in a row; and
that a call whose netlist has a bad pin (NaN result) leaves the shared scratch
clean for the next call.  The file sorts last so that a run stopping at the
first failure has already run every other test; it also passes alone in a
fresh process.
"""
import numpy as np
import pytest

import oracle
from paper_2511_10073_gb300 import netgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _placement(nl, seed):
    rng = np.random.default_rng(seed)
    xl, yl, xh, yh = nl.region
    xy = np.stack([rng.uniform(xl, xh, nl.num_cells), rng.uniform(yl, yh, nl.num_cells)], 1)
    return xy.astype(np.float32)


@pytest.mark.parametrize("cfg,seed", [("tiny", 3), ("medium", 2)])
def test_noalloc_hpwl_matches_workspace_hpwl_and_oracle(cfg, seed):
    import paper_2511_10073_gb300 as pl
    nl = netgen.make_netlist(cfg, seed)
    dnl = pl.DeviceNetlist(nl)
    xy = _placement(nl, seed)
    t = torch.tensor(xy.reshape(-1), device="cuda")
    ref = torch.zeros(1, dtype=torch.float64, device="cuda")
    pl.pl_hpwl(dnl, t, ref, pl.hpwl_workspace(nl.num_nets))
    want = oracle.hpwl(nl, xy[:, 0].astype(np.float64), xy[:, 1].astype(np.float64))
    for _ in range(2):
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        pl.pl_hpwl_noalloc(dnl, t, out)
        torch.cuda.synchronize()
        assert out.item() == ref.item()
        assert out.item() == pytest.approx(want, rel=1e-5)


def test_noalloc_bad_pin_then_valid_call():
    import paper_2511_10073_gb300 as pl
    nl = netgen.make_netlist("tiny", 4)
    xy = _placement(nl, 4)
    t = torch.tensor(xy.reshape(-1), device="cuda")
    pins = np.array(nl.pin_cell, copy=True)
    pins[17] = nl.num_cells + 3  # not read by the kernel; the result becomes NaN
    bad = netgen.Netlist(nl.net_ptr, pins, nl.pin_dx, nl.pin_dy, nl.cell_w, nl.cell_h,
                         nl.cell_kind, nl.fixed_x, nl.fixed_y, nl.region)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    pl.pl_hpwl_noalloc(pl.DeviceNetlist(bad), t, out)
    torch.cuda.synchronize()
    assert np.isnan(out.item())
    dnl = pl.DeviceNetlist(nl)
    ref = torch.zeros(1, dtype=torch.float64, device="cuda")
    pl.pl_hpwl(dnl, t, ref, pl.hpwl_workspace(nl.num_nets))
    pl.pl_hpwl_noalloc(dnl, t, out)
    torch.cuda.synchronize()
    assert np.isfinite(out.item()) and out.item() == ref.item()
    assert pl.lib().pl_last_error() == b""
