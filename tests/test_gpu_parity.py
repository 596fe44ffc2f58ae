"""GPU parity: every step of the CUDA path against the FP64 oracle.

Inputs are the seeded synthetic netlists of netgen.  Where a step consumes
coordinates, both sides get the same FP32 node coordinates (the oracle's own
previous step rounded to FP32; no oracle input comes from the GPU), so each
step is checked on its own:
  * static graph (A1): CSR bit-exact (columns, stored weights, baseWeight);
  * area hints (A2/A3): topology bit-exact (row pointers, columns, bins),
    D_b / C_b / phi_b bit-exact (FP64), hint weights bit-exact (FP32 and BF16
    storage), degrees and lambda_up within 1e-12 relative;
  * filters (A0, A4) and the whole initializer: coordinates within 1e-4 of the
    die width;
  * HPWL (A5): within 1e-5 relative.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2511_10073_gb300 import netgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def pl():
    import paper_2511_10073_gb300 as m
    return m


def cfg_params(name, **kw):
    base = dict(tiny=dict(nbx=16, nby=16), micro=dict(nbx=4, nby=4), small=dict(nbx=8, nby=8, det_ratio=0.4),
                medium=dict(nbx=32, nby=32), large=dict(nbx=32, nby=32))[name]
    base.update(kw)
    return base


class Side:
    """One netlist on both sides."""

    def __init__(self, nl, **kw):
        self.nl = nl
        self.kw = kw
        self.prm = pl().params(**kw)
        self.dnl = pl().DeviceNetlist(nl)
        self.g = pl().pl_build_graph(self.dnl, self.prm)
        self.info = self.g.info()
        self.o = oracle.Oracle(nl, **kw)
        self.N = self.info["N"]
        self.die = nl.region[2] - nl.region[0]

    def oracle_signal(self, seed):
        """The oracle's initial signal (A0 step 1) and its GiFt output, each
        rounded to FP32 (device tensors): the common input of both sides'
        next step."""
        ox, oy = self.o.init_signal(seed)
        a0 = np.stack([ox, oy], 1).astype(np.float32)
        gx, gy = self.o.gift(a0[:, 0].astype(np.float64), a0[:, 1].astype(np.float64))
        a1 = np.stack([gx, gy], 1).astype(np.float32)
        dev = lambda a: torch.tensor(a.reshape(-1), device="cuda")
        return dev(a0), dev(a1)


def to_np(t):
    return t.view(-1, 2).double().cpu().numpy()


# Degrees and lambda_up: the summed weights are bit-identical on both sides;
# the GPU adds them in double-float (about 48 significant bits, a few units of
# 2^-48 of the running sum per addition), the oracle in FP64.
DEG_REL = 1e-12


# -------------------------------------------------------------- A1 static
@pytest.mark.parametrize("cfg,seed,wd,perm", [
    ("micro", 1, 1, False), ("small", 1, 1, False), ("small", 2, 2, True),
    ("tiny", 1, 1, False), ("tiny", 3, 2, False), ("medium", 1, 1, False)])
def test_static_graph_bitexact(cfg, seed, wd, perm):
    nl = netgen.make_netlist(cfg, seed)
    if perm:
        nl = netgen.permuted(nl, 9)
    s = Side(nl, **cfg_params(cfg, wdtype=wd))
    ge = s.g.export_static()
    oe = s.o.static_csr()
    assert (s.info["macro_pins"], s.info["stars"], s.info["macros"]) == (s.o.Pm, s.o.S, s.o.Mm)
    assert np.array_equal(ge["rp"], oe["rp"])
    assert np.array_equal(ge["col"], oe["col"])
    assert np.array_equal(ge["w"], oe["w_store"])
    assert np.array_equal(ge["base_w"], oe["base_w"])


@pytest.mark.parametrize("wd", [1, 2])
def test_static_graph_hub_cells(wd):
    # cells with more than 128 static entries (hub rows summed by a whole
    # warp, one with over a thousand), repeated nets (summed lattice values
    # that need a division), star nets through the hub cells, and many small
    # nets around them
    rng = np.random.default_rng(11)
    cells = 4000
    nets = []
    for h, reps in [(0, 90), (1, 12), (2, 9), (3, 30)]:
        for _ in range(reps):
            nets.append(np.r_[h, rng.choice(np.arange(10, cells), 15, replace=False)])
    nets += [nets[3], nets[3], nets[100], nets[101]]  # parallel edges
    for h in (0, 2):
        nets.append(np.r_[h, rng.choice(np.arange(10, cells), 40, replace=False)])
    for _ in range(6000):
        nets.append(rng.choice(cells, rng.integers(2, 5), replace=False))
    ptr = np.r_[0, np.cumsum([len(n) for n in nets])].astype(np.int64)
    pins = np.concatenate(nets).astype(np.int32)
    z = np.zeros(len(pins), np.float32)
    nl = netgen.Netlist(ptr, pins, z, z, np.ones(cells, np.float32), np.ones(cells, np.float32),
                        np.zeros(cells, np.uint8), np.zeros(cells, np.float32),
                        np.zeros(cells, np.float32), (0.0, 0.0, 100.0, 100.0))
    s = Side(nl, **cfg_params("tiny", wdtype=wd))
    ge = s.g.export_static()
    oe = s.o.static_csr()
    lens = np.diff(oe["rp"])
    assert lens[:4].min() > 128 and lens[0] > 1000  # the hub cells
    assert np.array_equal(ge["rp"], oe["rp"])
    assert np.array_equal(ge["col"], oe["col"])
    assert np.array_equal(ge["w"], oe["w_store"])
    assert np.array_equal(ge["base_w"], oe["base_w"])


# -------------------------------------------------------- A2/A3 hints
def _compare_hints(s, ge, oe):
    """Augmented graph of one hint build against the oracle's: bins, D_b, C_b,
    phi_b, row pointers, columns and stored weights bit-identical (FP32 and
    BF16 storage both round the FP64 weight of the definition once); signed
    degrees within DEG_REL of the row's sum of |w|, lambda_up within DEG_REL."""
    assert np.array_equal(ge["cell_bin"], oe["cell_bin"])
    assert np.array_equal(ge["Db"], oe["Db"])
    assert np.array_equal(ge["Cb"], oe["Cb"])
    assert np.array_equal(ge["phi"], oe["phi"])
    assert np.array_equal(ge["rp"], oe["rp"])
    assert np.array_equal(ge["col"], oe["col"])
    bad = ge["w"] != oe["w"]
    assert not bad.any(), f"{bad.sum()} weights differ, e.g. {ge['w'][bad][:5]} vs {oe['w'][bad][:5]}"
    rp = oe["rp"]
    absw = np.bincount(np.repeat(np.arange(s.N), np.diff(rp)), weights=np.abs(oe["w"]),
                       minlength=s.N)
    derr = np.abs(ge["deg"] - oe["deg"])
    assert (derr <= DEG_REL * absw + 1e-300).all(), float((derr / np.maximum(absw, 1e-300)).max())
    assert abs(ge["lam_up"] - oe["lam_up"]) <= DEG_REL * abs(oe["lam_up"])
    return float((derr / np.maximum(absw, 1e-300)).max())


@pytest.mark.parametrize("cfg,seed,kw", [
    ("micro", 1, {}), ("small", 1, {}), ("small", 3, dict(wdtype=2)), ("tiny", 1, {}),
    ("tiny", 2, dict(nbx=32, nby=32)), ("tiny", 4, dict(nbx=20, nby=12, det_ratio=0.3, wdtype=2)),
    # a 7 x 7 window (49 slots): the bin rows' degree sums take two groups of 32 slots
    ("tiny", 7, dict(nbx=32, nby=32, det_ratio=0.25, wdtype=2)),
    # 4608 buckets: too many for the per-warp counters, the bucket lists by warp turns
    ("tiny", 8, dict(nbx=48, nby=48)),
    ("medium", 2, {}),
    # more bin buckets than the tiled counting sort takes: atomic bucket
    # counts, sorted buckets, bin rows gathered by the hub-chunk kernel
    ("tiny", 6, dict(nbx=96, nby=80)), ("medium", 3, dict(nbx=100, nby=100, wdtype=2))])
def test_hints_crossfed(cfg, seed, kw):
    nl = netgen.make_netlist(cfg, seed)
    s = Side(nl, **cfg_params(cfg, **kw))
    _, xy = s.oracle_signal(seed)
    pl().pl_build_hints(s.g, s.prm, xy)
    ge = s.g.export()
    a = to_np(xy)
    s.o.build_hints(a[:, 0], a[:, 1])
    oe = s.o.merged()
    _compare_hints(s, ge, oe)


def test_hints_stacked_macros():
    # ten macros on one site: the cells on it overlap all ten, more than the
    # cell pass records per cell, so the round falls back to an atomic
    # scatter and a segmented sort of the macro lists
    nl = netgen.make_netlist("tiny", 5)
    kind = np.asarray(nl.cell_kind)
    cw, ch = np.asarray(nl.cell_w), np.asarray(nl.cell_h)
    macros = np.flatnonzero(kind == netgen.KIND_MACRO)
    m = int(macros[np.argmax(cw[macros] * ch[macros])])
    rep = lambda a: np.r_[np.asarray(a), np.repeat(np.asarray(a)[m], 9)].astype(np.asarray(a).dtype)
    nl2 = netgen.Netlist(nl.net_ptr, nl.pin_cell, nl.pin_dx, nl.pin_dy, rep(nl.cell_w), rep(nl.cell_h),
                         rep(nl.cell_kind), rep(nl.fixed_x), rep(nl.fixed_y), nl.region)
    s = Side(nl2, **cfg_params("tiny"))
    _, xy = s.oracle_signal(5)
    # put a block of cells on the stacked site
    a = to_np(xy)
    movable = np.flatnonzero(kind == netgen.KIND_MOVABLE)[:200]
    rng = np.random.default_rng(5)
    fx, fy = float(np.asarray(nl.fixed_x)[m]), float(np.asarray(nl.fixed_y)[m])
    a[movable, 0] = fx + rng.uniform(-0.4, 0.4, len(movable)) * cw[m]
    a[movable, 1] = fy + rng.uniform(-0.4, 0.4, len(movable)) * ch[m]
    t = torch.tensor(a.astype(np.float32).reshape(-1), device="cuda")
    pl().pl_build_hints(s.g, s.prm, t)
    ge = s.g.export()
    b = to_np(t)
    s.o.build_hints(b[:, 0], b[:, 1])
    oe = s.o.merged()
    _compare_hints(s, ge, oe)


# ------------------------------------------------------------ A0 / A4
@pytest.mark.parametrize("cfg,seed,kw", [
    ("micro", 2, {}), ("small", 1, {}), ("tiny", 1, {}), ("tiny", 2, dict(wdtype=2)),
    ("tiny", 3, dict(gift_center=1, gift_k=(3, 1, 0), gift_sigma=(1.5, 3.0, 3.0))),
    # a sigma whose only band has k = 0, after the chain with steps
    ("tiny", 4, dict(gift_center=1, gift_k=(3, 1, 0), gift_sigma=(1.5, 1.5, 3.0))),
    # three chains with steps: one alone, then a pair of unequal lengths
    ("tiny", 5, dict(gift_k=(2, 3, 1), gift_sigma=(1.0, 2.0, 3.0), gift_alpha=(0.5, 0.3, 0.2))),
    # a pair of equal lengths, two bands sharing the last step of one chain
    ("small", 3, dict(gift_center=1, gift_k=(2, 2, 2), gift_sigma=(4.0, 2.0, 4.0), wdtype=2)),
    # one chain only
    ("tiny", 6, dict(gift_k=(1, 3, 2), gift_sigma=(2.0, 2.0, 2.0))),
    ("medium", 1, {})])
def test_init_and_gift_crossfed(cfg, seed, kw):
    nl = netgen.make_netlist(cfg, seed)
    s = Side(nl, **cfg_params(cfg, **kw))
    xg = torch.empty(s.N * 2, dtype=torch.float32, device="cuda")
    pl().pl_init_signal(s.g, seed, None, xg)
    ag = to_np(xg)
    ox, oy = s.o.init_signal(seed)
    mov = nl.cell_kind == 0
    C = nl.num_cells
    assert np.array_equal(ag[:C, 0][mov], ox[:C][mov].astype(np.float32))
    assert np.abs(ag[:, 0] - ox).max() <= 1e-6 * s.die
    x0, _ = s.oracle_signal(seed)
    x1 = torch.empty_like(x0)
    pl().pl_gift(s.g, s.prm, x0, x1)
    torch.cuda.synchronize()
    a0 = to_np(x0)
    gx, gy = s.o.gift(a0[:, 0], a0[:, 1])
    a1 = to_np(x1)
    err = max(np.abs(a1[:, 0] - gx).max(), np.abs(a1[:, 1] - gy).max())
    assert err <= 1e-4 * s.die, err


@pytest.mark.parametrize("cfg,seed,kw", [
    ("micro", 1, {}), ("small", 2, {}), ("tiny", 1, {}), ("tiny", 2, dict(wdtype=2)),
    ("tiny", 3, dict(ntaps=3, tap_k=(2, 4, 8, 0), tap_alpha=(1 / 3, 1 / 3, 1 / 3, 0))),
    ("tiny", 4, dict(pin_every_step=1, gamma=0.7)), ("tiny", 5, dict(nbx=32, nby=32)),
    ("medium", 3, {}), ("medium", 1, dict(wdtype=2, ntaps=3, tap_k=(2, 4, 8, 0),
                                         tap_alpha=(1 / 3, 1 / 3, 1 / 3, 0))),
    ("tiny", 6, dict(nbx=96, nby=80, wdtype=2)),
    # windows other than 3 x 3: 5 x 3 (15 slots) and 7 x 7 (49 slots, two groups
    # of 32 in the bin rows' sums), the chunk partials slot by slot
    ("tiny", 7, dict(nbx=20, nby=12, det_ratio=0.3, wdtype=2)),
    ("tiny", 8, dict(nbx=32, nby=32, det_ratio=0.25, wdtype=2, ntaps=3, tap_k=(2, 4, 8, 0),
                     tap_alpha=(1 / 3, 1 / 3, 1 / 3, 0)))])
def test_filter_step_crossfed(cfg, seed, kw):
    nl = netgen.make_netlist(cfg, seed)
    s = Side(nl, **cfg_params(cfg, **kw))
    _, xy = s.oracle_signal(seed)
    pl().pl_build_hints(s.g, s.prm, xy)
    out = torch.empty_like(xy)
    pl().pl_filter_apply(s.g, s.prm, xy, out)
    torch.cuda.synchronize()
    a = to_np(xy)
    s.o.build_hints(a[:, 0], a[:, 1])
    ox, oy = s.o.filter(a[:, 0], a[:, 1])
    b = to_np(out)
    err = max(np.abs(b[:, 0] - ox).max(), np.abs(b[:, 1] - oy).max())
    assert err <= 1e-4 * s.die, err


@pytest.mark.parametrize("cfg,seed,kw", [
    ("micro", 3, {}), ("small", 1, {}), ("tiny", 1, {}), ("tiny", 2, {}), ("tiny", 3, dict(wdtype=2)),
    ("tiny", 6, dict(gift_enable=0)), ("tiny", 7, dict(t_hint=0)), ("tiny", 8, dict(gamma=0.0))])
def test_full_initializer(cfg, seed, kw):
    nl = netgen.make_netlist(cfg, seed)
    s = Side(nl, **cfg_params(cfg, **kw))
    out = torch.empty(nl.num_cells * 2, dtype=torch.float32, device="cuda")
    pl().pl_filter_init(s.g, s.prm, seed, None, out)
    torch.cuda.synchronize()
    gx, gy = s.o.run(seed)
    b = to_np(out)
    C = nl.num_cells
    err = max(np.abs(b[:, 0] - gx[:C]).max(), np.abs(b[:, 1] - gy[:C]).max())
    assert err <= 1e-4 * s.die, err


def test_full_initializer_from_given_placement():
    nl = netgen.make_netlist("tiny", 9)
    s = Side(nl, **cfg_params("tiny"))
    rng = np.random.default_rng(0)
    xl, yl, xh, yh = nl.region
    xy0 = np.stack([rng.uniform(xl, xh, nl.num_cells), rng.uniform(yl, yh, nl.num_cells)], 1).astype(np.float32)
    t0 = torch.tensor(xy0.reshape(-1), device="cuda")
    out = torch.empty_like(t0)
    pl().pl_filter_init(s.g, s.prm, 0, t0, out)
    gx, gy = s.o.run(0, xy0=xy0.reshape(-1))
    b = to_np(out)
    err = max(np.abs(b[:, 0] - gx[:nl.num_cells]).max(), np.abs(b[:, 1] - gy[:nl.num_cells]).max())
    assert err <= 1e-4 * s.die


def test_full_initializer_net_through_every_cell():
    # one net through every cell (macros and I/O included): a star row of
    # every node, a star entry in every cell row, on top of a tiny netlist
    nl = netgen.make_netlist("tiny", 7)
    C = nl.num_cells
    z = np.zeros(C, np.float32)
    nl2 = netgen.Netlist(np.r_[nl.net_ptr, nl.net_ptr[-1] + C].astype(np.int64),
                         np.r_[nl.pin_cell, np.arange(C)].astype(np.int32),
                         np.r_[nl.pin_dx, z].astype(np.float32), np.r_[nl.pin_dy, z].astype(np.float32),
                         nl.cell_w, nl.cell_h, nl.cell_kind, nl.fixed_x, nl.fixed_y, nl.region)
    for wd in (1, 2):
        s = Side(nl2, **cfg_params("tiny", wdtype=wd))
        ge = s.g.export_static()
        oe = s.o.static_csr()
        assert np.array_equal(ge["col"], oe["col"]) and np.array_equal(ge["w"], oe["w_store"])
        assert np.array_equal(ge["base_w"], oe["base_w"])
        out = torch.empty(C * 2, dtype=torch.float32, device="cuda")
        pl().pl_filter_init(s.g, s.prm, 3, None, out)
        torch.cuda.synchronize()
        gx, gy = s.o.run(3)
        b = to_np(out)
        err = max(np.abs(b[:, 0] - gx[:C]).max(), np.abs(b[:, 1] - gy[:C]).max())
        assert err <= 1e-4 * s.die, err


# --------------------------------------------------------------- A5 HPWL
@pytest.mark.parametrize("cfg,seed", [("micro", 1), ("tiny", 2), ("medium", 1)])
def test_hpwl(cfg, seed):
    nl = netgen.make_netlist(cfg, seed)
    dnl = pl().DeviceNetlist(nl)
    rng = np.random.default_rng(seed)
    xl, yl, xh, yh = nl.region
    xy = np.stack([rng.uniform(xl, xh, nl.num_cells), rng.uniform(yl, yh, nl.num_cells)], 1).astype(np.float32)
    t = torch.tensor(xy.reshape(-1), device="cuda")
    ws = pl().hpwl_workspace(nl.num_nets)
    h = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(2):  # the second call reuses the workspace
        pl().pl_hpwl(dnl, t, h, ws)
        ref = oracle.hpwl(nl, xy[:, 0].astype(np.float64), xy[:, 1].astype(np.float64))
        assert h.item() == pytest.approx(ref, rel=1e-5)


def test_hpwl_big_nets_and_empty():
    cells = 100
    nl = netgen.Netlist(np.array([0, 0, 1, 41, 100], np.int64),
                        np.r_[np.arange(1), np.arange(40), np.arange(59) + 40].astype(np.int32) % cells,
                        np.zeros(100, np.float32), np.zeros(100, np.float32),
                        np.ones(cells, np.float32), np.ones(cells, np.float32),
                        np.zeros(cells, np.uint8), np.zeros(cells, np.float32),
                        np.zeros(cells, np.float32), (0.0, 0.0, 10.0, 10.0))
    xy = np.random.default_rng(1).uniform(0, 10, (cells, 2)).astype(np.float32)
    h = torch.zeros(1, dtype=torch.float64, device="cuda")
    pl().pl_hpwl(pl().DeviceNetlist(nl), torch.tensor(xy.reshape(-1), device="cuda"), h,
                 pl().hpwl_workspace(4))
    assert h.item() == pytest.approx(oracle.hpwl(nl, xy[:, 0], xy[:, 1]), rel=1e-6)


def test_hpwl_net_size_classes():
    # nets at every boundary of the kernel's classes (a lane up to 32 pins, a
    # warp up to 1024, a block beyond), the largest allowed net, spread over
    # the blocks' net ranges among many small nets
    rng = np.random.default_rng(7)
    cells = 40000
    sizes = rng.integers(0, 6, 3000)
    for pos, n in [(5, 32), (6, 33), (700, 1024), (701, 1025), (1500, 4097), (2200, 32768),
                   (2999, 2000), (0, 1500)]:
        sizes[pos] = n
    ptr = np.r_[0, np.cumsum(sizes)].astype(np.int64)
    pins = np.concatenate([rng.choice(cells, n, replace=False) for n in sizes]).astype(np.int32)
    dx = rng.uniform(-0.4, 0.4, len(pins)).astype(np.float32)
    dy = rng.uniform(-0.4, 0.4, len(pins)).astype(np.float32)
    nl = netgen.Netlist(ptr, pins, dx, dy, np.ones(cells, np.float32), np.ones(cells, np.float32),
                        np.zeros(cells, np.uint8), np.zeros(cells, np.float32),
                        np.zeros(cells, np.float32), (0.0, 0.0, 1000.0, 1000.0))
    xy = rng.uniform(0, 1000, (cells, 2)).astype(np.float32)
    h = torch.zeros(1, dtype=torch.float64, device="cuda")
    t = torch.tensor(xy.reshape(-1), device="cuda")
    pl().pl_hpwl(pl().DeviceNetlist(nl), t, h, pl().hpwl_workspace(len(sizes)))
    ref = oracle.hpwl(nl, xy[:, 0].astype(np.float64), xy[:, 1].astype(np.float64))
    assert h.item() == pytest.approx(ref, rel=1e-6)


# ------------------------------------------------------------ failures
def test_errors_are_reported():
    m = pl()
    nl = netgen.make_netlist("micro", 1)
    bad = netgen.Netlist(nl.net_ptr, nl.pin_cell.copy(), nl.pin_dx, nl.pin_dy, nl.cell_w,
                         nl.cell_h, nl.cell_kind, nl.fixed_x, nl.fixed_y, nl.region)
    bad.pin_cell[3] = nl.num_cells + 5
    with pytest.raises(m.PlError) as e:
        m.pl_build_graph(m.DeviceNetlist(bad), m.params(nbx=4, nby=4))
    assert e.value.code == m.PL_ERR_INVALID_ARG
    with pytest.raises(m.PlError) as e:
        m.pl_build_graph(m.DeviceNetlist(nl), m.params(nbx=4, nby=4, clique_max=40))
    assert e.value.code == m.PL_ERR_INVALID_ARG
    s = Side(nl, nbx=4, nby=4)
    xy = torch.full((s.N * 2,), float("nan"), device="cuda")
    with pytest.raises(m.PlError) as e:
        m.pl_build_hints(s.g, s.prm, xy)
    assert e.value.code == m.PL_ERR_NONFINITE
    with pytest.raises(m.PlError) as e:
        m.pl_build_hints(s.g, m.params(nbx=8, nby=4), xy)
    assert e.value.code == m.PL_ERR_INVALID_ARG
    ws = torch.empty(8, dtype=torch.uint8, device="cuda")
    with pytest.raises(m.PlError) as e:
        m.pl_hpwl(s.dnl, torch.zeros(nl.num_cells * 2, device="cuda"),
                  torch.zeros(1, dtype=torch.float64, device="cuda"), ws)
    assert e.value.code == m.PL_ERR_WORKSPACE


def test_empty_graph_spectrum_error():
    m = pl()
    cells = [(1.0, 1.0, 0, 0.0, 0.0)] * 3
    nl = netgen.Netlist(np.array([0, 1, 2], np.int64), np.array([0, 1], np.int32),
                        np.zeros(2, np.float32), np.zeros(2, np.float32),
                        np.ones(3, np.float32), np.ones(3, np.float32), np.zeros(3, np.uint8),
                        np.zeros(3, np.float32), np.zeros(3, np.float32), (0.0, 0.0, 10.0, 10.0))
    s = Side(nl, nbx=2, nby=2)
    x0, x1 = s.oracle_signal(1)
    with pytest.raises(m.PlError) as e:
        m.pl_build_hints(s.g, s.prm, x1)
    assert e.value.code == m.PL_ERR_SPECTRUM
    assert s.o.build_hints(*to_np(x1).T, check=False) == oracle.ERR_SPECTRUM


def test_rebuild_in_place_other_netlist():
    m = pl()
    a = netgen.make_netlist("tiny", 1)
    b = netgen.make_netlist("small", 2)
    prm = m.params(nbx=8, nby=8)
    g = m.pl_build_graph(m.DeviceNetlist(a), prm)
    g = m.pl_build_graph(m.DeviceNetlist(b), prm, graph=g)
    ge = g.export_static()
    oe = oracle.Oracle(b, nbx=8, nby=8).static_csr()
    assert np.array_equal(ge["col"], oe["col"]) and np.array_equal(ge["w"], oe["w_store"])


# ------------------------------------------- full size, as the benchmark runs it
LARGE = dict(nbx=32, nby=32, wdtype=2, ntaps=3, tap_k=(2, 4, 8, 0),
             tap_alpha=(1 / 3, 1 / 3, 1 / 3, 0))


def test_large_workload_steps_crossfed():
    """The 2.2M-cell workload in the benchmark's configuration: static graph
    and area-hint graph bit-exact (BF16 weights), one refinement round and
    HPWL against the oracle on the same FP32 input."""
    nl = netgen.make_netlist("large", 1)
    s = Side(nl, **LARGE)
    ge = s.g.export_static()
    oe = s.o.static_csr()
    assert np.array_equal(ge["rp"], oe["rp"]) and np.array_equal(ge["col"], oe["col"])
    assert np.array_equal(ge["w"], oe["w_store"]) and np.array_equal(ge["base_w"], oe["base_w"])
    del ge, oe
    x0, xy = s.oracle_signal(1)  # xy: the oracle's GiFt of x0, in FP32
    x1 = torch.empty_like(x0)
    pl().pl_gift(s.g, s.prm, x0, x1)
    a = to_np(xy)
    a1 = to_np(x1)
    assert np.abs(a1 - a).max() <= 1e-4 * s.die
    del x0, x1, a1
    pl().pl_build_hints(s.g, s.prm, xy)
    s.o.build_hints(a[:, 0], a[:, 1])
    _compare_hints(s, s.g.export(), s.o.merged())
    out = torch.empty_like(xy)
    pl().pl_filter_apply(s.g, s.prm, xy, out)
    ox, oy = s.o.filter(a[:, 0], a[:, 1])
    b = to_np(out)
    err = max(np.abs(b[:, 0] - ox).max(), np.abs(b[:, 1] - oy).max())
    assert err <= 1e-4 * s.die, err
    # HPWL of the oracle's round output, in FP32, on both sides
    c = np.stack([ox, oy], 1)[:nl.num_cells].astype(np.float32)
    cells = torch.tensor(c.reshape(-1), device="cuda")
    h = torch.zeros(1, dtype=torch.float64, device="cuda")
    pl().pl_hpwl(s.dnl, cells, h, pl().hpwl_workspace(nl.num_nets))
    ref = oracle.hpwl(nl, c[:, 0].astype(np.float64), c[:, 1].astype(np.float64))
    assert h.item() == pytest.approx(ref, rel=1e-5)
