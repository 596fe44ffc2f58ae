"""The OpenMP build of the oracle (timed as the all-cores CPU baseline)
returns the same bits as the single-threaded oracle the parity tests use."""
import numpy as np
import pytest

import oracle
from paper_2511_10073_gb300 import netgen


@pytest.mark.parametrize("cfg,kw", [
    ("tiny", dict(nbx=16, nby=16)),
    ("small", dict(nbx=8, nby=8, det_ratio=0.4, wdtype=oracle.W_BF16, ntaps=3,
                   tap_k=(2, 4, 8, 0), tap_alpha=(1 / 3, 1 / 3, 1 / 3, 0)))])
def test_parallel_oracle_is_bit_identical(cfg, kw, monkeypatch):
    monkeypatch.setenv("OMP_NUM_THREADS", "4")
    nl = netgen.make_netlist(cfg, 2)
    seq = oracle.Oracle(nl, **kw)
    par = oracle.Oracle(nl, parallel=True, **kw)
    sx, sy = seq.run(5)
    px, py = par.run(5)
    assert np.array_equal(sx, px) and np.array_equal(sy, py)
    a, b = seq.merged(), par.merged()
    for k in ("rp", "col", "w", "deg", "Db", "phi"):
        assert np.array_equal(a[k], b[k]), k
    assert a["lam_up"] == b["lam_up"]
    C = nl.num_cells
    assert oracle.hpwl(nl, sx[:C], sy[:C]) == oracle.hpwl(nl, px[:C], py[:C], parallel=True)
    assert oracle.host_cores() >= 1
