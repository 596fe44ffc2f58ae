"""Seeded synthetic mixed-size netlists.

This module only draws inputs: it holds none of the initializer's arithmetic
and is the one piece shared by the CUDA path's tests/benchmark and the CPU
oracle's tests.  The recipe stands in for the ISPD2005 / Ariane / BP Quad
benchmarks of the paper's evaluation (Sec. VIII, Table II), which are not
available: shapes follow Table II (movable std cells, fixed macros and I/Os,
nets about as many as cells) and the workload configurations below.

Recipe (units: site width = row height = 1):
  * std cells: w ~ U{1,2,3,4}, h = 1, movable (kind 0);
  * macros (kind 1, fixed): "area" mode draws area log-uniform in a stated
    range ([100, 1600] for the 2k-cell netlist) with aspect U[0.7, 1.4];
    "frac" mode draws relative areas log-uniform over a 10x range, scaled so
    all macros cover 40% of the die; placed without overlap by rejection
    sampling, largest first, on integer sites;
  * die: square; tiny: A_std/0.6 + A_macro, otherwise A_std/0.36 (std cells
    fill 60% of the area left by macros);
  * I/O pins (kind 2, fixed, w = h = 0): uniform on the die boundary, each
    attached to one random net;
  * macro pins: clamp(round(perimeter/8), 8, 64) per macro at uniform boundary
    sites, each joined to one random net;
  * net degree: 55% 2-pin, 20% 3-pin, 25% P(d) ~ d^-2.5 on [4, cap];
  * locality: a random recursive bisection of the std-cell index space into
    leaves of <= 32 cells; each net takes a uniform seed cell and draws every
    further pin from the seed's ancestor at level l with P(l) ~ 2^-l;
  * std-cell pin offsets uniform in the inner 80% of the cell.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

KIND_MOVABLE, KIND_MACRO, KIND_IO = 0, 1, 2

CONFIGS = {
    # name: std cells, macros, I/O, nets, degree cap, macro mode
    "micro": dict(n_std=28, n_macro=1, n_io=4, n_nets=36, cap=8, macro_mode="area",
                  macro_area=(9.0, 25.0)),
    "small": dict(n_std=300, n_macro=3, n_io=16, n_nets=330, cap=40, macro_mode="area",
                  macro_area=(25.0, 225.0)),
    "tiny": dict(n_std=2000, n_macro=20, n_io=64, n_nets=2200, cap=64, macro_mode="area",
                 macro_area=(100.0, 1600.0)),
    "medium": dict(n_std=210_000, n_macro=550, n_io=1000, n_nets=220_000, cap=2000, macro_mode="frac"),
    "half": dict(n_std=1_100_000, n_macro=4000, n_io=4000, n_nets=1_125_000, cap=5000, macro_mode="frac"),
    "large": dict(n_std=2_200_000, n_macro=8000, n_io=8000, n_nets=2_250_000, cap=10_000, macro_mode="frac"),
}


def batch_configs(seed: int, n: int = 64, lo: int = 5_000, hi: int = 500_000) -> list:
    """A batch of n designs of uneven size: std cells log-uniform in [lo, hi],
    macros 0.2-1% of the cells, I/O 0.5% (at least 16), nets 1.02 x the
    cells, the medium recipe's degree law (cap 2,000) and macro share."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(n):
        c = int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))
        out.append(dict(n_std=c, n_macro=max(1, int(round(c * rng.uniform(0.002, 0.01)))),
                        n_io=max(16, int(round(0.005 * c))), n_nets=int(round(1.02 * c)),
                        cap=2000, macro_mode="frac"))
    return out


@dataclass
class Netlist:
    net_ptr: np.ndarray    # int64[M+1]
    pin_cell: np.ndarray   # int32[P]
    pin_dx: np.ndarray     # float32[P] offset from cell centre
    pin_dy: np.ndarray     # float32[P]
    cell_w: np.ndarray     # float32[C]
    cell_h: np.ndarray     # float32[C]
    cell_kind: np.ndarray  # uint8[C]
    fixed_x: np.ndarray    # float32[C] centres, meaningful for kind != 0
    fixed_y: np.ndarray    # float32[C]
    region: tuple          # (xl, yl, xh, yh) as python floats
    name: str = ""

    @property
    def num_cells(self) -> int:
        return int(self.cell_w.shape[0])

    @property
    def num_nets(self) -> int:
        return int(self.net_ptr.shape[0] - 1)

    @property
    def num_pins(self) -> int:
        return int(self.pin_cell.shape[0])

    @property
    def num_movable(self) -> int:
        return int(np.count_nonzero(self.cell_kind == KIND_MOVABLE))

    def translated(self, dx: float, dy: float) -> "Netlist":
        """Same netlist with the region and every fixed object shifted."""
        fx = self.fixed_x.copy()
        fy = self.fixed_y.copy()
        fixed = self.cell_kind != KIND_MOVABLE
        fx[fixed] += np.float32(dx)
        fy[fixed] += np.float32(dy)
        xl, yl, xh, yh = self.region
        return Netlist(self.net_ptr, self.pin_cell, self.pin_dx, self.pin_dy, self.cell_w,
                       self.cell_h, self.cell_kind, fx, fy, (xl + dx, yl + dy, xh + dx, yh + dy),
                       self.name + "+t")


def _hierarchy(n: int, rng: np.random.Generator, leaf: int = 32):
    """Random recursive bisection of [0, n).  Returns (leaf_of[n], anc_lo, anc_hi)
    where anc_*[leaf_id, l] is the index range of that leaf's ancestor at level l
    (level 0 = the leaf itself; rows are padded with the root)."""
    leaves_lo, leaves_hi, leaves_anc = [], [], []
    stack = [(0, n, [])]
    while stack:
        lo, hi, anc = stack.pop()
        if hi - lo <= leaf:
            leaves_lo.append(lo)
            leaves_hi.append(hi)
            leaves_anc.append(anc)
            continue
        f = rng.uniform(0.4, 0.6)
        mid = lo + max(1, min(hi - lo - 1, int(round((hi - lo) * f))))
        nanc = anc + [(lo, hi)]
        stack.append((mid, hi, nanc))
        stack.append((lo, mid, nanc))
    depth = 1 + max(len(a) for a in leaves_anc)
    nl = len(leaves_lo)
    anc_lo = np.empty((nl, depth), np.int64)
    anc_hi = np.empty((nl, depth), np.int64)
    order = np.argsort(np.asarray(leaves_lo))
    leaf_of = np.empty(n, np.int64)
    for new_id, k in enumerate(order):
        lo, hi, anc = leaves_lo[k], leaves_hi[k], leaves_anc[k]
        chain = [(lo, hi)] + anc[::-1]
        chain += [(0, n)] * (depth - len(chain))
        anc_lo[new_id] = [c[0] for c in chain]
        anc_hi[new_id] = [c[1] for c in chain]
        leaf_of[lo:hi] = new_id
    return leaf_of, anc_lo, anc_hi


def _place_macros(w: np.ndarray, h: np.ndarray, side: float, rng: np.random.Generator):
    """Non-overlapping rejection sampling on integer sites, largest macro first.
    Returns lower-left corners (float64)."""
    n = w.shape[0]
    llx = np.zeros(n)
    lly = np.zeros(n)
    order = np.argsort(-(w * h), kind="stable")
    gsz = float(max(1.0, max(w.max(), h.max()) if n else 1.0))
    ng = int(math.ceil(side / gsz)) + 1
    grid: dict = {}
    isz = int(side)
    for k in order:
        wk, hk = w[k], h[k]
        placed = False
        for _attempt in range(20000):
            x0 = float(rng.integers(0, max(1, int(isz - wk) + 1)))
            y0 = float(rng.integers(0, max(1, int(isz - hk) + 1)))
            gx0, gx1 = int(x0 // gsz), int((x0 + wk) // gsz)
            gy0, gy1 = int(y0 // gsz), int((y0 + hk) // gsz)
            ok = True
            for gx in range(gx0, min(gx1, ng - 1) + 1):
                for gy in range(gy0, min(gy1, ng - 1) + 1):
                    for j in grid.get((gx, gy), ()):
                        if (x0 < llx[j] + w[j] and llx[j] < x0 + wk and
                                y0 < lly[j] + h[j] and lly[j] < y0 + hk):
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                llx[k], lly[k] = x0, y0
                for gx in range(gx0, min(gx1, ng - 1) + 1):
                    for gy in range(gy0, min(gy1, ng - 1) + 1):
                        grid.setdefault((gx, gy), []).append(k)
                placed = True
                break
        if not placed:
            raise RuntimeError("macro placement failed; die too crowded")
    return llx, lly


def _boundary_points(n: int, wid: float, hei: float, rng: np.random.Generator):
    """n points uniform on the boundary of a wid x hei rectangle, relative to its
    lower-left corner."""
    per = 2.0 * (wid + hei)
    t = rng.uniform(0.0, per, n)
    x = np.empty(n)
    y = np.empty(n)
    s0 = t < wid
    s1 = (t >= wid) & (t < wid + hei)
    s2 = (t >= wid + hei) & (t < 2 * wid + hei)
    s3 = t >= 2 * wid + hei
    x[s0], y[s0] = t[s0], 0.0
    x[s1], y[s1] = wid, t[s1] - wid
    x[s2], y[s2] = wid - (t[s2] - wid - hei), hei
    x[s3], y[s3] = 0.0, hei - (t[s3] - 2 * wid - hei)
    return x, y


def make_netlist(config: str | dict, seed: int, xl: float = 0.0, yl: float = 0.0) -> Netlist:
    """Draw one netlist.  `config` is a key of CONFIGS or a dict of the same form."""
    cfg = dict(CONFIGS[config]) if isinstance(config, str) else dict(config)
    name = config if isinstance(config, str) else "custom"
    rng = np.random.Generator(np.random.PCG64(seed))
    n_std, n_mac, n_io = cfg["n_std"], cfg["n_macro"], cfg["n_io"]
    n_nets, cap = cfg["n_nets"], cfg["cap"]

    std_w = rng.integers(1, 5, n_std).astype(np.float64)
    std_h = np.ones(n_std)
    a_std = float(std_w.sum())

    mode = cfg["macro_mode"]
    if mode == "area":
        lo, hi = cfg["macro_area"]
        area = np.exp(rng.uniform(math.log(lo), math.log(hi), n_mac))
        asp = rng.uniform(0.7, 1.4, n_mac)
        mw = np.maximum(1.0, np.round(np.sqrt(area * asp)))
        mh = np.maximum(1.0, np.round(np.sqrt(area / asp)))
        die_area = a_std / 0.6 + float((mw * mh).sum())
        side = float(math.ceil(math.sqrt(die_area)))
    else:
        die_area = a_std / 0.36
        side = float(math.ceil(math.sqrt(die_area)))
        rel = np.exp(rng.uniform(0.0, math.log(10.0), n_mac))
        area = rel / rel.sum() * 0.40 * side * side
        asp = rng.uniform(0.7, 1.4, n_mac)
        mw = np.maximum(1.0, np.round(np.sqrt(area * asp)))
        mh = np.maximum(1.0, np.round(np.sqrt(area / asp)))
    llx, lly = _place_macros(mw, mh, side, rng)

    C = n_std + n_mac + n_io
    cell_w = np.zeros(C, np.float32)
    cell_h = np.zeros(C, np.float32)
    kind = np.zeros(C, np.uint8)
    fx = np.zeros(C, np.float32)
    fy = np.zeros(C, np.float32)
    cell_w[:n_std], cell_h[:n_std] = std_w, std_h
    m0 = n_std
    cell_w[m0:m0 + n_mac], cell_h[m0:m0 + n_mac] = mw, mh
    kind[m0:m0 + n_mac] = KIND_MACRO
    fx[m0:m0 + n_mac] = xl + llx + mw / 2.0
    fy[m0:m0 + n_mac] = yl + lly + mh / 2.0
    i0 = n_std + n_mac
    kind[i0:] = KIND_IO
    iox, ioy = _boundary_points(n_io, side, side, rng)
    fx[i0:], fy[i0:] = xl + iox, yl + ioy

    # ---- net degrees
    u = rng.uniform(size=n_nets)
    deg = np.where(u < 0.55, 2, 3).astype(np.int64)
    tail = u >= 0.75
    support = np.arange(4, cap + 1, dtype=np.float64)
    pmf = support ** -2.5
    cdf = np.cumsum(pmf) / pmf.sum()
    deg[tail] = 4 + np.searchsorted(cdf, rng.uniform(size=int(tail.sum())), side="right")
    deg = np.minimum(deg, cap)

    # ---- std-cell pins with hierarchical locality
    leaf_of, anc_lo, anc_hi = _hierarchy(n_std, rng)
    depth = anc_lo.shape[1]
    seed_cell = rng.integers(0, n_std, n_nets)
    n_extra = int((deg - 1).sum())
    net_of_extra = np.repeat(np.arange(n_nets), deg - 1)
    lvl_p = 2.0 ** -np.arange(depth)
    lvl_cdf = np.cumsum(lvl_p) / lvl_p.sum()
    lvl = np.searchsorted(lvl_cdf, rng.uniform(size=n_extra), side="right")
    lvl = np.minimum(lvl, depth - 1)
    lf = leaf_of[seed_cell[net_of_extra]]
    lo_r = anc_lo[lf, lvl]
    hi_r = anc_hi[lf, lvl]
    extra_cell = lo_r + np.floor(rng.uniform(size=n_extra) * (hi_r - lo_r)).astype(np.int64)
    extra_cell = np.minimum(extra_cell, hi_r - 1)

    pin_net = np.concatenate([np.arange(n_nets), net_of_extra])
    pin_cell = np.concatenate([seed_cell, extra_cell])
    pdx = (rng.uniform(size=pin_cell.shape[0]) - 0.5) * 0.8 * std_w[pin_cell]
    pdy = (rng.uniform(size=pin_cell.shape[0]) - 0.5) * 0.8 * std_h[pin_cell]

    # ---- macro pins on the macro boundary, each joins a random net
    mp_net, mp_cell, mp_dx, mp_dy = [], [], [], []
    for k in range(n_mac):
        npin = int(min(64, max(8, round(2.0 * (mw[k] + mh[k]) / 8.0))))
        bx, by = _boundary_points(npin, mw[k], mh[k], rng)
        mp_dx.append(bx - mw[k] / 2.0)
        mp_dy.append(by - mh[k] / 2.0)
        mp_cell.append(np.full(npin, m0 + k))
        mp_net.append(rng.integers(0, n_nets, npin))
    if n_mac:
        pin_net = np.concatenate([pin_net] + mp_net)
        pin_cell = np.concatenate([pin_cell] + mp_cell)
        pdx = np.concatenate([pdx] + mp_dx)
        pdy = np.concatenate([pdy] + mp_dy)
    # ---- I/O pins
    io_net = rng.integers(0, n_nets, n_io)
    pin_net = np.concatenate([pin_net, io_net])
    pin_cell = np.concatenate([pin_cell, np.arange(i0, C)])
    pdx = np.concatenate([pdx, np.zeros(n_io)])
    pdy = np.concatenate([pdy, np.zeros(n_io)])

    # group pins by net, shuffled inside each net
    order = np.lexsort((rng.uniform(size=pin_net.shape[0]), pin_net))
    pin_net = pin_net[order]
    net_ptr = np.zeros(n_nets + 1, np.int64)
    np.cumsum(np.bincount(pin_net, minlength=n_nets), out=net_ptr[1:])
    return Netlist(net_ptr=net_ptr,
                   pin_cell=pin_cell[order].astype(np.int32),
                   pin_dx=pdx[order].astype(np.float32),
                   pin_dy=pdy[order].astype(np.float32),
                   cell_w=cell_w, cell_h=cell_h, cell_kind=kind, fixed_x=fx, fixed_y=fy,
                   region=(float(xl), float(yl), float(xl + side), float(yl + side)),
                   name=f"{name}/s{seed}")


def permuted(nl: Netlist, seed: int) -> Netlist:
    """The same circuit with cells renumbered and nets reordered (tests that
    nothing depends on std cells, macros and I/Os coming in blocks)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    C = nl.num_cells
    perm = rng.permutation(C)           # new id -> old id
    inv = np.empty(C, np.int64)
    inv[perm] = np.arange(C)
    M = nl.num_nets
    norder = rng.permutation(M)
    deg = np.diff(nl.net_ptr)
    new_ptr = np.zeros(M + 1, np.int64)
    np.cumsum(deg[norder], out=new_ptr[1:])
    idx = np.concatenate([np.arange(nl.net_ptr[e], nl.net_ptr[e + 1]) for e in norder]) \
        if M else np.zeros(0, np.int64)
    return Netlist(net_ptr=new_ptr,
                   pin_cell=inv[nl.pin_cell[idx]].astype(np.int32),
                   pin_dx=nl.pin_dx[idx], pin_dy=nl.pin_dy[idx],
                   cell_w=nl.cell_w[perm], cell_h=nl.cell_h[perm], cell_kind=nl.cell_kind[perm],
                   fixed_x=nl.fixed_x[perm], fixed_y=nl.fixed_y[perm], region=nl.region,
                   name=nl.name + "+perm")
