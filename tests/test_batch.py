"""The batched serving form (pl_filter_init_batch): a batch of designs of
uneven size initialized concurrently on several streams gives each design the
same bits as its own pl_filter_init call, and the designs' results pass the
oracle's check."""
import numpy as np
import pytest

import oracle
from paper_2511_10073_gb300 import netgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_batch_equals_single_runs():
    import paper_2511_10073_gb300 as pl
    cfgs = netgen.batch_configs(5, n=7, lo=300, hi=30_000)
    nls = [netgen.make_netlist(c, 40 + i) for i, c in enumerate(cfgs)]
    prm = pl.params(nbx=16, nby=16, wdtype=pl.PL_W_BF16, ntaps=3, tap_k=(2, 4, 8, 0),
                    tap_alpha=(1 / 3, 1 / 3, 1 / 3, 0))
    dnls = [pl.DeviceNetlist(nl) for nl in nls]
    graphs = [pl.pl_build_graph(d, prm) for d in dnls]
    seeds = [11 + i for i in range(len(nls))]
    single = []
    for g, nl, sd in zip(graphs, nls, seeds):
        o = torch.empty(nl.num_cells * 2, dtype=torch.float32, device="cuda")
        pl.pl_filter_init(g, prm, sd, None, o)
        single.append(o)
    torch.cuda.synchronize()
    # both forms, several stream counts and short-row CTA counts: the same bits
    for union, ns, rc in ((0, 1, 5), (0, 3, 5), (1, 1, 5), (1, 3, 3), (1, 4, 1)):
        outs = [torch.full_like(o, float("nan")) for o in single]
        streams = [torch.cuda.Stream() for _ in range(ns)]
        pl.pl_filter_init_batch(graphs, prm, seeds, outs, streams,
                                pl.batch_opts(union_products=union, rows_ctas_per_sm=rc))
        torch.cuda.synchronize()
        for a, b in zip(single, outs):
            assert torch.equal(a, b), (union, ns, rc)
    # the autotuner runs every candidate and leaves the same bits
    outs = [torch.full_like(o, float("nan")) for o in single]
    best, ms = pl.pl_batch_autotune(graphs, prm, seeds, outs, [torch.cuda.Stream() for _ in range(4)])
    torch.cuda.synchronize()
    assert ms > 0 and best.streams in (1, 2, 4) and best.union_products in (0, 1)
    for a, b in zip(single, outs):
        assert torch.equal(a, b)
    # the smallest design against the oracle
    i = int(np.argmin([nl.num_cells for nl in nls]))
    o = oracle.Oracle(nls[i], nbx=16, nby=16, wdtype=oracle.W_BF16, ntaps=3, tap_k=(2, 4, 8, 0),
                      tap_alpha=(1 / 3, 1 / 3, 1 / 3, 0))
    gx, gy = o.run(seeds[i])
    xy = single[i].view(-1, 2).double().cpu().numpy()
    C = nls[i].num_cells
    die = nls[i].region[2] - nls[i].region[0]
    err = max(np.abs(xy[:, 0] - gx[:C]).max(), np.abs(xy[:, 1] - gy[:C]).max())
    assert err <= 1e-4 * die, err


def test_batch_reports_the_failing_design():
    import paper_2511_10073_gb300 as pl
    nl = netgen.make_netlist("micro", 1)
    prm = pl.params(nbx=4, nby=4)
    g = pl.pl_build_graph(pl.DeviceNetlist(nl), prm)
    out = torch.empty(nl.num_cells * 2, dtype=torch.float32, device="cuda")
    with pytest.raises(pl.PlError) as e:  # per-design form: the failing design is named
        pl.pl_filter_init_batch([g, g], pl.params(nbx=8, nby=4), [1, 2], [out, out],
                                [torch.cuda.Stream()], pl.batch_opts(union_products=0))
    assert e.value.code == pl.PL_ERR_INVALID_ARG and "design" in str(e.value)
    with pytest.raises(pl.PlError) as e:  # union form: checked before any work
        pl.pl_filter_init_batch([g, g], pl.params(nbx=8, nby=4), [1, 2], [out, out],
                                [torch.cuda.Stream()])
    assert e.value.code == pl.PL_ERR_INVALID_ARG
    with pytest.raises(pl.PlError) as e:  # union form: workspace too small
        pl.pl_filter_init_batch([g, g], prm, [1, 2], [out, out], [torch.cuda.Stream()],
                                ws=torch.empty(256, dtype=torch.uint8, device="cuda"))
    assert e.value.code == pl.PL_ERR_WORKSPACE
