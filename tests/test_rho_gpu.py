"""GPU parity of the macro charge-density schedules (Sec. VI): the per-bin
integrals of pl_macro_density against the FP64 oracle, for the four models
at several iterations of the schedule, on the macros of a synthetic netlist
(1e-11 relative for the FP64 models, 1e-6 for the two whose point values the
GPU takes in FP32)."""
import numpy as np
import pytest

import oracle
from paper_2511_10073_gb300 import netgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _macros(cfg, seed):
    nl = netgen.make_netlist(cfg, seed)
    m = np.flatnonzero(np.asarray(nl.cell_kind) == netgen.KIND_MACRO)
    return nl, [np.asarray(a, np.float32)[m] for a in (nl.fixed_x, nl.fixed_y, nl.cell_w, nl.cell_h)]


@pytest.mark.parametrize("cfg,nb", [("tiny", (16, 16)), ("medium", (64, 48))])
@pytest.mark.parametrize("model", [0, 1, 2, 3])
def test_macro_density_matches_oracle(cfg, nb, model):
    import paper_2511_10073_gb300 as pl
    nl, geo = _macros(cfg, 2)
    dev = [torch.tensor(a, device="cuda") for a in geo]
    nbx, nby = nb
    rp = pl.rho_params(model=model)
    orp = oracle.rho_params(model=model)
    for f in ("T", "r0", "r1", "beta_min", "beta_max", "alpha0", "alpha1", "sigma_factor",
              "k_factor", "panels", "nodes"):
        assert getattr(rp, f) == getattr(orp, f), f
    out = torch.empty(nbx * nby, dtype=torch.float64, device="cuda")
    for t in (0, 1, 45, 150, 299, 300):
        pl.pl_macro_density(rp, t, *dev, nl.region, nbx, nby, out)
        got = out.cpu().numpy()
        ref = oracle.macro_density(orp, t, *(a.astype(np.float64) for a in geo), nl.region, nbx, nby)
        abin = (nl.region[2] - nl.region[0]) * (nl.region[3] - nl.region[1]) / (nbx * nby)
        # FP64 throughout for the Gaussian and exponential-like models; the
        # radial models' point values are FP32 (about 1e-7 relative each)
        tol = 1e-11 if model in (0, 1) else 1e-6
        assert np.allclose(got, ref, rtol=tol, atol=tol * abin), (t, np.abs(got - ref).max())
        if model == 0 or t == 300:  # every macro's full charge inside the region
            assert got.sum() == pytest.approx(float((geo[2].astype(np.float64) * geo[3]).sum()), rel=1e-9)


def test_macro_density_rejects_bad_schedule():
    import paper_2511_10073_gb300 as pl
    out = torch.empty(4, dtype=torch.float64, device="cuda")
    z = torch.zeros(1, device="cuda")
    with pytest.raises(pl.PlError) as e:
        pl.pl_macro_density(pl.rho_params(), 301, z, z, z + 1, z + 1, (0, 0, 2, 2), 2, 2, out)
    assert e.value.code == pl.PL_ERR_INVALID_ARG
    with pytest.raises(pl.PlError):
        pl.pl_macro_density(pl.rho_params(nodes=40), 3, z, z, z + 1, z + 1, (0, 0, 2, 2), 2, 2, out)
