"""Pins of the FP64 oracle to things other than itself.

Every check here compares the oracle with mathematics the paper fixes
(closed-form filter responses on ring and path graphs, the Gershgorin bound,
Laplacian invariants, the Schur complement of the star model), with brute
force written independently on tiny inputs (dense matrices, exact fractions),
with the C library or numpy (exp, rounding), or with published test vectors
(splitmix64).  No CUDA code is involved.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2511_10073_gb300 import netgen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ helpers
def make(cells, nets, region, pins_offsets=None):
    """cells: list of (w, h, kind, fx, fy); nets: list of lists of cell ids
    (or (cell, dx, dy) tuples)."""
    cw = np.array([c[0] for c in cells], np.float32)
    ch = np.array([c[1] for c in cells], np.float32)
    kind = np.array([c[2] for c in cells], np.uint8)
    fx = np.array([c[3] for c in cells], np.float32)
    fy = np.array([c[4] for c in cells], np.float32)
    ptr = [0]
    pc, pdx, pdy = [], [], []
    for n in nets:
        for p in n:
            if isinstance(p, tuple):
                pc.append(p[0]); pdx.append(p[1]); pdy.append(p[2])
            else:
                pc.append(p); pdx.append(0.0); pdy.append(0.0)
        ptr.append(len(pc))
    return netgen.Netlist(np.array(ptr, np.int64), np.array(pc, np.int32),
                          np.array(pdx, np.float32), np.array(pdy, np.float32),
                          cw, ch, kind, fx, fy, tuple(float(v) for v in region), "custom")


def ring_netlist(n, path=False):
    cells = [(1.0, 1.0, 0, 0.0, 0.0) for _ in range(n)]
    nets = [[i, (i + 1) % n] for i in range(n if not path else n - 1)]
    return make(cells, nets, (0.0, 0.0, float(n), 1.0))


def ulps(a, b):
    return abs(a - b) / math.ulp(b) if b != 0 else abs(a)


def dense_from_csr(rp, col, w, n):
    A = np.zeros((n, n))
    for i in range(n):
        for k in range(rp[i], rp[i + 1]):
            A[i, col[k]] += w[k]
    return A


def brute_static(nl, clique_max=16):
    """Independent statement of the instance graph: node of each pin, distinct
    node sets, exact Fraction weights, dense."""
    C = nl.num_cells
    pin_node = []
    nmp = 0
    for p in range(nl.num_pins):
        c = int(nl.pin_cell[p])
        if nl.cell_kind[c] == netgen.KIND_MACRO:
            pin_node.append(C + nmp)
            nmp += 1
        else:
            pin_node.append(c)
    sets = [sorted(set(pin_node[nl.net_ptr[e]:nl.net_ptr[e + 1]])) for e in range(nl.num_nets)]
    nstar = sum(1 for s in sets if len(s) > clique_max)
    Nst = C + nmp + nstar
    W = [dict() for _ in range(Nst)]
    s_id = C + nmp
    for s in sets:
        p = len(s)
        if p < 2:
            continue
        if p <= clique_max:
            for a in s:
                for b in s:
                    if a != b:
                        W[a][b] = W[a].get(b, Fraction(0)) + Fraction(1, p - 1)
        else:
            for a in s:
                W[a][s_id] = Fraction(p, p - 1)
                W[s_id][a] = Fraction(p, p - 1)
            s_id += 1
    return pin_node, sets, W, nmp, nstar


# ---------------------------------------------------------- scalar kernels
def test_exp_within_one_ulp_of_libm():
    rng = np.random.default_rng(0)
    xs = np.concatenate([rng.uniform(-60, 60, 20000), rng.uniform(-1, 1, 5000),
                         [0.0, -0.0, 1e-300, -1e-300, 0.5, -0.5, 1.0, -1.0, 700.0, -700.0,
                          -708.5, -740.0, 709.5]])
    worst = 0.0
    for x in xs:
        ref = math.exp(float(x))
        got = oracle.exp(float(x))
        if ref == 0.0:
            assert got == 0.0
            continue
        worst = max(worst, ulps(got, ref))
    assert worst <= 1.0, worst
    assert oracle.exp(0.0) == 1.0
    assert oracle.exp(-1000.0) == 0.0
    assert math.isinf(oracle.exp(1000.0))
    assert math.isnan(oracle.exp(float("nan")))


def test_splitmix64_published_vector():
    vals = [int(l) for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))
            if l.strip() and not l.startswith("#")]
    for k, v in enumerate(vals):
        u = oracle.u01(1234567, k)
        assert u * 2.0 ** 53 == float(v >> 11)
        assert 0.0 <= u < 1.0


def _bf16_brute(w):
    """Nearest bfloat16 (ties to even) by examining the neighbouring bf16 bit
    patterns with exact rational distances."""
    if w == 0.0:
        return w
    f = np.float32(w)
    if np.isinf(f):
        f = np.float32(np.copysign(np.finfo(np.float32).max, w))
    bits = int(np.array([f], np.float32).view(np.uint32)[0]) & 0xFFFF0000
    best = None
    for d in (-0x10000, 0, 0x10000, 0x20000):
        b = (bits + d) & 0xFFFFFFFF
        if (b >> 16) & 0x7F80 == 0x7F80:  # inf/nan patterns
            cand = math.copysign(math.inf, w)
            dist = math.inf
        else:
            cand = float(np.array([b], np.uint32).view(np.float32)[0])
            if math.copysign(1.0, cand) != math.copysign(1.0, w) and cand != 0.0:
                continue
            dist = abs(Fraction(cand) - Fraction(w))
        key = (dist, (b >> 16) & 1)
        if best is None or key < best[0]:
            best = (key, cand)
    return best[1]


def test_store_rounding_matches_brute_force():
    rng = np.random.default_rng(1)
    vals = list(rng.standard_normal(3000) * np.exp(rng.uniform(-80, 80, 3000)))
    # exact ties between two bf16 values, both parities
    for m in (1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -(1.0 + 2 ** -8), 1.5 + 2 ** -8):
        vals.append(m)
    vals += [1e-39, 3e-40, -2e-41, 1.1754943508222875e-38, 3.3e38, -3.39e38]
    for w in vals:
        w = float(w)
        assert oracle.store(w, oracle.W_FP32) == float(np.float32(w))
        assert oracle.store(w, oracle.W_FP64) == w
        got = oracle.store(w, oracle.W_BF16)
        exp_ = _bf16_brute(w)
        assert got == exp_ or (math.isinf(got) and math.isinf(exp_)), (w, got, exp_)


# ------------------------------------------------------- A1 static graph
@pytest.mark.parametrize("cfg,seed,perm", [("micro", 1, False), ("micro", 2, False),
                                           ("small", 1, False), ("small", 3, True)])
def test_static_graph_equals_dense_brute_force(cfg, seed, perm):
    nl = netgen.make_netlist(cfg, seed)
    if perm:
        nl = netgen.permuted(nl, 5)
    o = oracle.Oracle(nl, nbx=4, nby=4, wdtype=oracle.W_BF16)
    pin_node, sets, W, nmp, nstar = brute_static(nl)
    assert (o.Pm, o.S) == (nmp, nstar)
    st = o.static_csr()
    nodes = o.nodes()
    assert np.array_equal(nodes["pin_node"], np.array(pin_node, np.int32))
    rp, col, we, ws = st["rp"], st["col"], st["w_exact"], st["w_store"]
    for i in range(o.Nst):
        cols = list(col[rp[i]:rp[i + 1]])
        assert cols == sorted(W[i].keys())
        for k, j in enumerate(cols):
            assert we[rp[i] + k] == float(W[i][j])          # correctly rounded exact sum
            assert ws[rp[i] + k] == _bf16_brute(float(W[i][j]))
    for i in range(o.C):
        # baseWeight: the correctly rounded sum of the row's weights over their count
        row = we[rp[i]:rp[i + 1]]
        want = math.fsum(row) / len(row) if len(row) else 0.0
        assert st["base_w"][i] == want
    # fixed positions of macro pin nodes: macro centre + pin offset
    for p, v in enumerate(pin_node):
        if v >= o.C:
            c = nl.pin_cell[p]
            assert nodes["fx"][v] == float(nl.fixed_x[c]) + float(nl.pin_dx[p])
            assert nodes["nkind"][v] == 2


def test_weighted_degree_identity_medium_size():
    nl = netgen.make_netlist("tiny", 4)
    o = oracle.Oracle(nl, nbx=16, nby=16, wdtype=oracle.W_FP64)
    st = o.static_csr()
    _, sets, _, _, _ = brute_static(nl)
    want = 0.0
    for s in sets:
        p = len(s)
        if 2 <= p <= 16:
            want += p                       # p(p-1) ordered pairs of weight 1/(p-1)
        elif p > 16:
            want += 2.0 * p * p / (p - 1)   # 2p entries of weight p/(p-1)
    assert math.fsum(st["w_exact"]) == pytest.approx(want, rel=1e-12)


def test_star_model_schur_complement_is_clique():
    p = 21
    cells = [(1.0, 1.0, 0, 0.0, 0.0) for _ in range(p)]
    nl = make(cells, [list(range(p))], (0, 0, 50, 50))
    o = oracle.Oracle(nl, nbx=2, nby=2, wdtype=oracle.W_FP64)
    assert o.S == 1
    st = o.static_csr()
    W = dense_from_csr(st["rp"], st["col"], st["w_exact"], o.Nst)
    L = np.diag(W.sum(1)) - W
    a = list(range(p))
    s = [o.Nst - 1]
    Lab = L[np.ix_(a, a)] - L[np.ix_(a, s)] @ np.linalg.inv(L[np.ix_(s, s)]) @ L[np.ix_(s, a)]
    Wc = np.full((p, p), 1.0 / (p - 1))
    np.fill_diagonal(Wc, 0.0)
    Lc = np.diag(Wc.sum(1)) - Wc
    assert np.abs(Lab - Lc).max() < 1e-12


def test_degenerate_nets_are_skipped():
    cells = [(1.0, 1.0, 0, 0.0, 0.0) for _ in range(4)] + [(0.0, 0.0, 2, 0.0, 3.0)]
    nets = [[], [0], [1, 1, 1], [2, 3, 3, 2], [4, 0]]
    o = oracle.Oracle(make(cells, nets, (0, 0, 10, 10)), nbx=2, nby=2, wdtype=oracle.W_FP64)
    st = o.static_csr()
    W = dense_from_csr(st["rp"], st["col"], st["w_exact"], o.Nst)
    want = np.zeros_like(W)
    want[2, 3] = want[3, 2] = 1.0
    want[4, 0] = want[0, 4] = 1.0
    assert np.array_equal(W, want)


def test_invalid_inputs_rejected():
    cells = [(1.0, 1.0, 0, 0.0, 0.0) for _ in range(3)]
    with pytest.raises(oracle.OracleError):
        oracle.Oracle(make(cells, [[0, 5]], (0, 0, 10, 10)))        # pin on a missing cell
    with pytest.raises(oracle.OracleError):
        oracle.Oracle(make(cells, [[0, 1]], (0, 0, 0, 10)))         # empty region
    bad = make([(0.0, 2.0, 1, 5.0, 5.0)] + cells, [[0, 1]], (0, 0, 10, 10))
    with pytest.raises(oracle.OracleError):
        oracle.Oracle(bad)                                          # zero-width macro


# ------------------------------------------------------------ A2 hints
def test_hint_weights_hand_computed():
    # one 20x10 macro at (50, 50); movable cells joined in pairs by 2-pin nets
    # (baseWeight 1); one bin covering the die (window 1x1)
    cells = [(20.0, 10.0, 1, 50.0, 50.0),
             (2.0, 1.0, 0, 0, 0), (2.0, 1.0, 0, 0, 0),   # A, B
             (1.0, 1.0, 0, 0, 0), (1.0, 1.0, 0, 0, 0)]   # C, D
    nets = [[1, 2], [3, 4]]
    nl = make(cells, nets, (0.0, 0.0, 100.0, 100.0))
    o = oracle.Oracle(nl, nbx=1, nby=1, wdtype=oracle.W_FP64, mu=4.0, capacity=1.0)
    gx = np.zeros(o.N); gy = np.zeros(o.N)
    pos = {1: (55.0, 52.0), 2: (80.0, 80.0), 3: (40.9, 54.9), 4: (50.0, 55.6)}
    for c, (x, y) in pos.items():
        gx[c], gy[c] = x, y
    o.build_hints(gx, gy)
    m = o.merged()
    Nst = o.Nst
    vm, vb = Nst, Nst + 1
    # bin: area of movable cells 2+2+1+1 = 6; capacity (1e4 - 200)/1e4
    Db = 6.0 / 1e4
    Cb = (1.0 * (1e4 - 200.0)) / 1e4
    assert m["Db"][0] == Db and m["Cb"][0] == Cb
    phi = 2.0 / (1.0 + math.exp(-4.0 * (Db - Cb))) - 1.0
    assert m["phi"][0] == pytest.approx(phi, rel=1e-15)
    assert phi < 0  # underfull bin: attractive edges
    W = dense_from_csr(m["rp"], m["col"], m["w"], o.N)
    # macro edges: A overlaps (|dx|=5 < 11, |dy|=2 < 5.5); C overlaps
    # (|dx|=9.1 < 10.5, |dy|=4.9 < 5.5); B no; D: |dy|=5.6 >= 5.5 no
    assert W[1, vm] == pytest.approx(-math.exp(-max(5.0 / 10.0, 2.0 / 5.0)), rel=1e-15)
    assert W[3, vm] == pytest.approx(-math.exp(-max(9.1 / 10.0, 4.9 / 5.0)), rel=1e-15)
    assert W[2, vm] == 0.0 and W[4, vm] == 0.0
    for c, (x, y) in pos.items():
        r = max(abs(x - 50.0) / 50.0, abs(y - 50.0) / 50.0)
        assert W[c, vb] == pytest.approx(-(math.exp(-r) * phi) * 1.0, rel=1e-15)
    assert np.array_equal(W, W.T)
    # virtual rows list cells ascending
    assert list(m["col"][m["rp"][vm]:m["rp"][vm + 1]]) == [1, 3]
    assert list(m["col"][m["rp"][vb]:m["rp"][vb + 1]]) == [1, 2, 3, 4]


def test_phi_sign_and_zero_at_capacity():
    # region n x 1, n unit cells, one bin: D_b = 1 = C_b exactly -> phi = 0
    nl = ring_netlist(8)
    o = oracle.Oracle(nl, nbx=1, nby=1, wdtype=oracle.W_FP64, capacity=1.0)
    gx = np.zeros(o.N); gy = np.full(o.N, 0.5)
    gx[:8] = np.arange(8) + 0.5
    o.build_hints(gx, gy)
    assert o.merged()["phi"][0] == 0.0
    for cap, sign in ((0.5, 1.0), (2.0, -1.0)):     # overfull -> phi > 0, underfull -> < 0
        o2 = oracle.Oracle(nl, nbx=1, nby=1, wdtype=oracle.W_FP64, capacity=cap)
        o2.build_hints(gx, gy)
        m = o2.merged()
        assert np.sign(m["phi"][0]) == sign
        wb = m["w"][m["rp"][0]:m["rp"][1]][-1]       # cell 0's bin edge
        assert np.sign(wb) == -sign                   # repulsive when overfull


def test_hint_structure_matches_numpy_statement():
    nl = netgen.make_netlist("small", 2)
    nb = 16
    o = oracle.Oracle(nl, nbx=nb, nby=nb, det_ratio=0.2, wdtype=oracle.W_FP64)
    assert (o.hx, o.hy) == (1, 1)
    rng = np.random.default_rng(3)
    xl, yl, xh, yh = nl.region
    gx, gy = o.init_signal(9)
    mov = nl.cell_kind == 0
    gx[:o.C][mov] = rng.uniform(xl, xh, mov.sum())
    gy[:o.C][mov] = rng.uniform(yl, yh, mov.sum())
    o.build_hints(gx, gy)
    m = o.merged()
    bw = o.static_csr()["base_w"]
    wb, hb = (xh - xl) / nb, (yh - yl) / nb
    # integer decisions in FP32: bin = floor((x - xl) * (nb / (xh - xl)))
    f32 = np.float32
    bxs = np.clip(np.floor((gx[:o.C].astype(f32) - f32(xl)) * f32(nb / (xh - xl))), 0, nb - 1).astype(int)
    bys = np.clip(np.floor((gy[:o.C].astype(f32) - f32(yl)) * f32(nb / (yh - yl))), 0, nb - 1).astype(int)
    area = nl.cell_w.astype(np.float64) * nl.cell_h
    Db = np.zeros(nb * nb)
    for i in np.where(mov)[0]:
        Db[bys[i] * nb + bxs[i]] += area[i]
    assert np.allclose(m["Db"], Db / (wb * hb), rtol=1e-14, atol=0)
    assert np.array_equal(m["cell_bin"][mov], (bys * nb + bxs)[mov])
    macros = np.where(nl.cell_kind == 1)[0]
    st = o.static_csr()
    for i in np.where(mov)[0]:
        row_c = m["col"][m["rp"][i]:m["rp"][i + 1]]
        row_w = m["w"][m["rp"][i]:m["rp"][i + 1]]
        ns = st["rp"][i + 1] - st["rp"][i]
        hc, hw = list(row_c[ns:]), list(row_w[ns:])
        want_c, want_w = [], []
        if bw[i] > 0:
            for k, c in enumerate(macros):
                dxf = abs(f32(gx[i]) - nl.fixed_x[c])
                dyf = abs(f32(gy[i]) - nl.fixed_y[c])
                if dxf < f32(0.5) * (nl.cell_w[i] + nl.cell_w[c]) and \
                        dyf < f32(0.5) * (nl.cell_h[i] + nl.cell_h[c]):
                    dx, dy = abs(gx[i] - float(nl.fixed_x[c])), abs(gy[i] - float(nl.fixed_y[c]))
                    want_c.append(o.Nst + k)
                    r = max(dx / (nl.cell_w[c] * 0.5), dy / (nl.cell_h[c] * 0.5))
                    want_w.append(-(np.exp(-r) * bw[i]))
            for yy in range(bys[i] - 1, bys[i] + 2):
                for xx in range(bxs[i] - 1, bxs[i] + 2):
                    if 0 <= xx < nb and 0 <= yy < nb:
                        b = yy * nb + xx
                        want_c.append(o.Nst + o.Mm + b)
                        xb, yb = xl + (xx + 0.5) * wb, yl + (yy + 0.5) * hb
                        r = max(abs(gx[i] - xb) / (wb * 0.5), abs(gy[i] - yb) / (hb * 0.5))
                        want_w.append(-(np.exp(-r) * m["phi"][b] * bw[i]))
        assert hc == want_c
        assert np.allclose(hw, want_w, rtol=4e-16 * 4, atol=0)


def test_bin_density_blocked_sum_order():
    """D_b adds cell areas in blocks of 64 (hint cells first, then the others,
    each ascending); with areas that are not exactly summable the blocked
    order is visible, and it must match an independent statement of it."""
    n = 200
    cells = [(float(1.0 + (k % 7) * 0.1), float(1.0 + (k % 5) * 0.013), 0, 0.0, 0.0)
             for k in range(n)] + [(1.0, 1.0, 0, 0.0, 0.0)]
    # cells 100, 101 and n have no net (baseWeight 0): they come last
    nets = [[k, k + 1] for k in range(0, n, 2) if k != 100]
    nl = make(cells, nets, (0.0, 0.0, 10.0, 10.0))
    o = oracle.Oracle(nl, nbx=1, nby=1, wdtype=oracle.W_FP64)
    gx, gy = o.init_signal(1)
    o.build_hints(gx, gy)
    areas = [float(np.float32(c[0])) * float(np.float32(c[1])) for c in cells]
    nonhint = [100, 101, n]
    seq = [areas[k] for k in range(n + 1) if k not in nonhint] + [areas[k] for k in nonhint]

    def bsum(a):
        if len(a) <= 64:
            s = 0.0
            for v in a:
                s += v
            return s
        return bsum([bsum(a[j:j + 64]) for j in range(0, len(a), 64)])

    assert o.merged()["Db"][0] == bsum(seq) / 100.0
    assert abs(bsum(seq) - math.fsum(seq)) < 1e-12 * math.fsum(seq)


def test_nonfinite_coordinates_rejected():
    nl = netgen.make_netlist("micro", 1)
    o = oracle.Oracle(nl, nbx=4, nby=4)
    gx, gy = o.init_signal(1)
    gx[0] = np.nan
    assert o.build_hints(gx, gy, check=False) == oracle.ERR_NONFINITE


def test_empty_graph_has_no_spectrum():
    cells = [(1.0, 1.0, 0, 0, 0) for _ in range(3)]
    o = oracle.Oracle(make(cells, [[0], [1]], (0, 0, 10, 10)), nbx=2, nby=2)
    gx, gy = o.init_signal(1)
    assert o.build_hints(gx, gy, check=False) == oracle.ERR_SPECTRUM


# ------------------------------------------------------ A3 signed Laplacian
def test_signed_laplacian_invariants_and_gershgorin():
    nl = netgen.make_netlist("small", 1)
    o = oracle.Oracle(nl, nbx=8, nby=8, det_ratio=0.4, wdtype=oracle.W_FP32)
    gx, gy = o.run(3)
    o.build_hints(gx, gy)
    m = o.merged()
    W = dense_from_csr(m["rp"], m["col"], m["w"], o.N)
    assert np.array_equal(W, W.T)
    assert (W < 0).any()
    absw = np.abs(W).sum(1)
    for i in range(o.N):
        assert abs(m["deg"][i] - math.fsum(W[i])) <= 1e-13 * max(absw[i], 1e-300)
    L = np.diag(m["deg"]) - W
    assert np.abs(L.sum(1)).max() <= 1e-12 * absw.max()
    ev = np.linalg.eigvalsh(L)
    assert ev.max() <= m["lam_up"] * (1 + 1e-12)
    assert m["lam_up"] == pytest.approx(max(m["deg"] + absw), rel=1e-14)


# ------------------------------------------------------- A4 refinement filter
def _setup_small():
    nl = netgen.make_netlist("small", 2)
    o = oracle.Oracle(nl, nbx=8, nby=8, det_ratio=0.4, wdtype=oracle.W_FP32)
    gx, gy = o.run(5)
    o.build_hints(gx, gy)
    return nl, o, gx, gy


def test_filter_equals_dense_power_and_spectral_form():
    nl, o, gx, gy = _setup_small()
    m = o.merged()
    W = dense_from_csr(m["rp"], m["col"], m["w"], o.N)
    L = np.diag(m["deg"]) - W
    lam = m["lam_up"]
    P = (lam * np.eye(o.N) - L) / lam
    for k in (1, 2, 5, 8):
        want = np.linalg.matrix_power(P, k) @ gx
        got = o.hr_steps(k, gx)
        assert np.abs(got - want).max() <= 1e-9 * max(1.0, np.abs(want).max())
    ev, U = np.linalg.eigh(L)
    h = (1.0 - ev / lam) ** 8
    want = U @ (h * (U.T @ gy))
    got = o.hr_steps(8, gy)
    assert np.abs(got - want).max() <= 1e-8 * max(1.0, np.abs(want).max())
    ones = np.ones(o.N)
    assert np.abs(o.hr_steps(8, ones) - 1.0).max() < 1e-10


@pytest.mark.parametrize("path", [False, True])
def test_refinement_filter_closed_form_ring_and_path(path):
    n = 24
    nl = ring_netlist(n, path=path)
    o = oracle.Oracle(nl, nbx=1, nby=1, wdtype=oracle.W_FP64, capacity=1.0)
    gx = np.zeros(o.N); gy = np.full(o.N, 0.5)
    gx[:n] = np.arange(n) + 0.5
    o.build_hints(gx, gy)
    m = o.merged()
    assert m["lam_up"] == 4.0 and m["phi"][0] == 0.0
    i = np.arange(n)
    for j in (1, 3, 7, 12):
        for k in (1, 3, 8):
            x = np.zeros(o.N)
            if path:
                x[:n] = np.cos(np.pi * j * (i + 0.5) / n)
                resp = np.cos(np.pi * j / (2 * n)) ** (2 * k)
            else:
                th = 2 * np.pi * j / n
                x[:n] = np.cos(th * i)
                resp = np.cos(th / 2) ** (2 * k)
            y = o.hr_steps(k, x)
            assert np.abs(y[:n] - resp * x[:n]).max() < 1e-13


def test_filter_step_relax_repin_clamp():
    nl, o, gx, gy = _setup_small()
    nodes = o.nodes()
    fixed = nodes["nkind"] == 2
    # gamma = 0: identity on an in-region signal
    o0 = oracle.Oracle(nl, nbx=8, nby=8, det_ratio=0.4, gamma=0.0)
    o0.build_hints(gx, gy)
    ox, oy = o0.filter(gx, gy)
    assert np.array_equal(ox, gx) and np.array_equal(oy, gy)
    # one tap of order k with weight 1, gamma g: (1-g) x + g H^k x, re-pinned, clamped
    g = 0.3
    o1 = oracle.Oracle(nl, nbx=8, nby=8, det_ratio=0.4, gamma=g, clamp=0,
                       tap_k=(5, 0, 0, 0))
    o1.build_hints(gx, gy)
    hx = o1.hr_steps(5, gx)
    hx[fixed] = nodes["fx"][fixed]
    want = (1 - g) * gx + g * hx
    want[fixed] = nodes["fx"][fixed]
    ox, _ = o1.filter(gx, gy)
    assert np.abs(ox - want).max() < 1e-12 * np.abs(want).max()
    # taps: alpha-weighted sum of powers
    o2 = oracle.Oracle(nl, nbx=8, nby=8, det_ratio=0.4, gamma=1.0, clamp=0, ntaps=3,
                       tap_k=(2, 4, 8, 0), tap_alpha=(0.2, 0.3, 0.5, 0.0))
    o2.build_hints(gx, gy)
    want = 0.2 * o2.hr_steps(2, gy) + 0.3 * o2.hr_steps(4, gy) + 0.5 * o2.hr_steps(8, gy)
    want[fixed] = nodes["fy"][fixed]
    _, oy = o2.filter(gx, gy)
    assert np.abs(oy - want).max() < 1e-10 * np.abs(want).max()
    # clamping keeps movable cells inside the region
    xl, yl, xh, yh = nl.region
    ox, oy = o.filter(gx * 3.0 - 100.0, gy)
    mov = nodes["nkind"] != 2
    assert (ox[mov] >= xl + nodes["hw"][mov] - 1e-12).all()
    assert (ox[mov] <= xh - nodes["hw"][mov] + 1e-12).all()
    assert np.array_equal(ox[fixed], nodes["fx"][fixed])


def test_pin_every_step_keeps_fixed_nodes():
    nl, o, gx, gy = _setup_small()
    o1 = oracle.Oracle(nl, nbx=8, nby=8, det_ratio=0.4, pin_every_step=1, gamma=1.0,
                       clamp=0, tap_k=(2, 0, 0, 0))
    o1.build_hints(gx, gy)
    nodes = o1.nodes()
    fixed = nodes["nkind"] == 2
    one = o1.hr_steps(1, gx)
    one[fixed] = nodes["fx"][fixed]
    two = o1.hr_steps(1, one)
    two[fixed] = nodes["fx"][fixed]
    ox, _ = o1.filter(gx, gy)
    assert np.abs(ox - two).max() < 1e-12 * np.abs(two).max()


# --------------------------------------------------------------- A0 GiFt
def test_gift_band_closed_form_on_ring():
    n = 20
    nl = ring_netlist(n)
    o = oracle.Oracle(nl, nbx=1, nby=1)
    i = np.arange(n)
    for sigma in (2.0, 4.0):
        for j in (0, 2, 5, 10):
            th = 2 * np.pi * j / n
            x = np.zeros(o.N)
            x[:n] = np.cos(th * i)
            for k in (1, 2, 4):
                y = o.gift_band(sigma, k, x)
                resp = ((2 * np.cos(th) + sigma) / (2 + sigma)) ** k
                assert np.abs(y[:n] - resp * x[:n]).max() < 1e-13


def test_gift_band_dense_and_multiband():
    nl = netgen.make_netlist("small", 1)
    o = oracle.Oracle(nl, nbx=4, nby=4, wdtype=oracle.W_BF16)
    st = o.static_csr()
    A = np.zeros((o.N, o.N))
    A[:o.Nst, :o.Nst] = dense_from_csr(st["rp"], st["col"], st["w_store"], o.Nst)
    rng = np.random.default_rng(0)
    x = rng.uniform(0, 50, o.N)
    for sigma, k in ((2.0, 2), (4.0, 4)):
        d = A.sum(1) + sigma
        At = (A + sigma * np.eye(o.N)) / np.sqrt(np.outer(d, d))
        want = np.linalg.matrix_power(At, k) @ x
        assert np.abs(o.gift_band(sigma, k, x) - want).max() < 1e-10 * np.abs(want).max()
    # the three bands, re-pinned and clamped
    gx, gy = o.init_signal(4)
    ox, _ = o.gift(gx, gy)
    nodes = o.nodes()
    fixed = nodes["nkind"] == 2
    want = sum(a * o.gift_band(s, k, gx) for a, s, k in
               zip((0.7, 0.2, 0.1), (4.0, 4.0, 2.0), (4, 2, 2)))
    want[fixed] = nodes["fx"][fixed]
    xl, _, xh, _ = nl.region
    mov = ~fixed
    want[mov] = np.clip(want[mov], xl + nodes["hw"][mov], xh - nodes["hw"][mov])
    assert np.abs(ox - want).max() < 1e-10 * np.abs(want).max()


def test_init_signal_definition():
    nl = netgen.make_netlist("small", 1)
    o = oracle.Oracle(nl, nbx=4, nby=4)
    gx, gy = o.init_signal(77)
    xl, yl, xh, yh = nl.region
    nodes = o.nodes()
    for i in range(0, o.C, 37):
        if nl.cell_kind[i] == 0:
            assert gx[i] == xl + oracle.u01(77, 2 * i) * (xh - xl)
            assert gy[i] == yl + oracle.u01(77, 2 * i + 1) * (yh - yl)
        else:
            assert gx[i] == nl.fixed_x[i]
    _, sets, _, _, _ = brute_static(nl)
    stars = [s for s in sets if len(s) > 16]
    for k, s in enumerate(stars):
        v = o.C + o.Pm + k
        assert gx[v] == pytest.approx(math.fsum(gx[s]) / len(s), rel=1e-15)
    assert np.array_equal(gx[nodes["nkind"] == 2], nodes["fx"][nodes["nkind"] == 2])


# ------------------------------------------------------------------ A5 HPWL
def test_hpwl_hand_and_brute_force():
    cells = [(1.0, 1.0, 0, 0, 0), (1.0, 1.0, 0, 0, 0), (0.0, 0.0, 2, 7.0, 9.0)]
    nets = [[(0, 0.25, -0.5), (1, -0.25, 0.0)], [(2, 0.0, 0.0)], [], [0, 1, 2]]
    nl = make(cells, nets, (0, 0, 10, 10))
    cx = np.array([1.0, 4.0, 7.0]); cy = np.array([2.0, 6.0, 9.0])
    want = (abs((1.0 + 0.25) - (4.0 - 0.25)) + abs((2.0 - 0.5) - 6.0)) + 0.0 + (6.0 + 7.0)
    assert oracle.hpwl(nl, cx, cy) == want
    nl = netgen.make_netlist("small", 3)
    rng = np.random.default_rng(2)
    cx = rng.uniform(0, 50, nl.num_cells); cy = rng.uniform(0, 50, nl.num_cells)
    tot = []
    for e in range(nl.num_nets):
        px = [cx[nl.pin_cell[k]] + nl.pin_dx[k] for k in range(nl.net_ptr[e], nl.net_ptr[e + 1])]
        py = [cy[nl.pin_cell[k]] + nl.pin_dy[k] for k in range(nl.net_ptr[e], nl.net_ptr[e + 1])]
        if px:
            tot.append(max(px) - min(px) + max(py) - min(py))
    assert oracle.hpwl(nl, cx, cy) == pytest.approx(math.fsum(tot), rel=1e-13)


# ------------------------------------------------------------- whole path
def test_translation_equivariance_centered():
    nl = netgen.make_netlist("tiny", 2)
    nt = nl.translated(64.0, -32.0)
    a = oracle.Oracle(nl, nbx=16, nby=16, gift_center=1)
    b = oracle.Oracle(nt, nbx=16, nby=16, gift_center=1)
    ax, ay = a.run(11)
    bx, by = b.run(11)
    die = nl.region[2] - nl.region[0]
    # the shifted float32 fixed positions round by up to one float32 ulp
    assert np.abs((bx - 64.0) - ax).max() < 1e-6 * die
    assert np.abs((by + 32.0) - ay).max() < 1e-6 * die


def test_zero_iterations_and_zero_relaxation():
    nl = netgen.make_netlist("tiny", 1)
    a = oracle.Oracle(nl, nbx=16, nby=16, t_hint=0)
    gx, gy = a.init_signal(3)
    fx, fy = a.gift(gx, gy)
    rx, ry = a.run(3)
    assert np.array_equal(rx, fx) and np.array_equal(ry, fy)
    b = oracle.Oracle(nl, nbx=16, nby=16, gamma=0.0)
    bx, by = b.run(3)
    assert np.array_equal(bx, fx) and np.array_equal(by, fy)


def _overlap(nl, cx, cy):
    mov = nl.cell_kind == 0
    tot = 0.0
    for m in np.where(nl.cell_kind == 1)[0]:
        ox = np.minimum(cx[mov] + nl.cell_w[mov] / 2, nl.fixed_x[m] + nl.cell_w[m] / 2) - \
            np.maximum(cx[mov] - nl.cell_w[mov] / 2, nl.fixed_x[m] - nl.cell_w[m] / 2)
        oy = np.minimum(cy[mov] + nl.cell_h[mov] / 2, nl.fixed_y[m] + nl.cell_h[m] / 2) - \
            np.maximum(cy[mov] - nl.cell_h[mov] / 2, nl.fixed_y[m] - nl.cell_h[m] / 2)
        tot += float(np.sum(np.clip(ox, 0, None) * np.clip(oy, 0, None)))
    return tot


def test_refinement_reduces_macro_overlap_on_most_seeds():
    """Qualitative claim of the ablation (Sec. VIII-B): area hints move cells
    off macros compared with the GSP initialization alone."""
    wins = 0
    seeds = range(1, 11)
    for s in seeds:
        nl = netgen.make_netlist("tiny", s)
        g0 = oracle.Oracle(nl, nbx=16, nby=16, t_hint=0).run(s)
        g3 = oracle.Oracle(nl, nbx=16, nby=16, t_hint=3).run(s)
        C = nl.num_cells
        wins += _overlap(nl, g3[0][:C], g3[1][:C]) < _overlap(nl, g0[0][:C], g0[1][:C])
    assert wins >= 8
