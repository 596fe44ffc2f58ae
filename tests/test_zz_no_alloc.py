"""The allocation-free HPWL entry point (pl_hpwl_noalloc).

Some callers cannot allocate device memory or pass scratch to a library (a
host framework that owns every device allocation, a path where allocating is
not allowed); pl_hpwl_noalloc serves them with a fixed scratch array inside
the library.  This file checks it through the C ABI against pl_hpwl, on two
calls in a row.  It sorts last so that a run stopping at the first failure has
already run every other test; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from paper_2511_10073_gb300 import netgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cfg,seed", [("tiny", 3), ("medium", 2)])
def test_noalloc_hpwl_matches_workspace_hpwl(cfg, seed):
    import paper_2511_10073_gb300 as pl
    nl = netgen.make_netlist(cfg, seed)
    dnl = pl.DeviceNetlist(nl)
    rng = np.random.default_rng(seed)
    xl, yl, xh, yh = nl.region
    xy = np.stack([rng.uniform(xl, xh, nl.num_cells), rng.uniform(yl, yh, nl.num_cells)], 1)
    t = torch.tensor(xy.astype(np.float32).reshape(-1), device="cuda")
    ref = torch.zeros(1, dtype=torch.float64, device="cuda")
    pl.pl_hpwl(dnl, t, ref, pl.hpwl_workspace(nl.num_nets))
    for _ in range(2):
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        pl.pl_hpwl_noalloc(dnl, t, out)
        torch.cuda.synchronize()
        assert out.item() == pytest.approx(ref.item(), rel=1e-5)
