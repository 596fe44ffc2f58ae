"""FP64 CPU oracle of the area-hint refinement initializer (arXiv 2511.10073).

TEST INFRASTRUCTURE ONLY.  The C code in orc.c is the plain, sequential FP64
statement of the method; this module loads it with ctypes and moves numpy
arrays in and out.  Only the tests, the smoke check and the benchmark's CPU
baseline may import it.  It imports nothing from the CUDA package.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liborc.so")
_SO_OMP = os.path.join(_HERE, "liborc_omp.so")
_SRC = os.path.join(_HERE, "orc.c")

W_FP64, W_FP32, W_BF16 = 0, 1, 2
ERR_INVALID, ERR_SPECTRUM, ERR_NONFINITE = 1, 5, 6

# Parameter readings (Table I names; values where the paper gives none).
DEFAULTS = dict(
    clique_max=16, wdtype=W_FP32, gift_enable=1, gift_center=0,
    gift_k=(4, 2, 2), gift_sigma=(4.0, 4.0, 2.0), gift_alpha=(0.7, 0.2, 0.1),
    t_hint=3, nbx=32, nby=32, gamma=0.5, det_ratio=0.1, capacity=1.0, mu=4.0,
    ntaps=1, tap_k=(8, 0, 0, 0), tap_alpha=(1.0, 0.0, 0.0, 0.0),
    pin_every_step=0, clamp=1,
)


def _compile(so: str, extra: list, force: bool) -> str:
    if force or not os.path.exists(so) or os.path.getmtime(so) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "orc.h"))):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               *extra, "-shared", "-o", so + ".tmp", _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(so + ".tmp", so)
    return so


def build(force: bool = False) -> str:
    """Compile orc.c into liborc.so next to it (single-threaded, no FMA
    contraction): the oracle every test compares with."""
    return _compile(_SO, [], force)


def build_parallel(force: bool = False) -> str:
    """The same source built with OpenMP (liborc_omp.so): its parallel loops
    write disjoint outputs with unchanged arithmetic, so it returns the same
    bits as liborc.so.  Used only to time the oracle on all host cores."""
    return _compile(_SO_OMP, ["-fopenmp"], force)


def host_cores() -> int:
    """Host cores this process may run on (the OpenMP build's thread count)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class _Netlist(C.Structure):
    _fields_ = [("num_cells", C.c_int32), ("num_nets", C.c_int32), ("num_pins", C.c_int64),
                ("net_ptr", C.c_void_p), ("pin_cell", C.c_void_p),
                ("pin_dx", C.c_void_p), ("pin_dy", C.c_void_p),
                ("cell_w", C.c_void_p), ("cell_h", C.c_void_p), ("cell_kind", C.c_void_p),
                ("fixed_x", C.c_void_p), ("fixed_y", C.c_void_p),
                ("xl", C.c_double), ("yl", C.c_double), ("xh", C.c_double), ("yh", C.c_double)]


class _Params(C.Structure):
    _fields_ = [("clique_max", C.c_int32), ("wdtype", C.c_int32),
                ("gift_enable", C.c_int32), ("gift_center", C.c_int32),
                ("gift_k", C.c_int32 * 3), ("gift_sigma", C.c_double * 3),
                ("gift_alpha", C.c_double * 3), ("t_hint", C.c_int32),
                ("nbx", C.c_int32), ("nby", C.c_int32),
                ("gamma", C.c_double), ("det_ratio", C.c_double), ("capacity", C.c_double),
                ("mu", C.c_double), ("ntaps", C.c_int32), ("tap_k", C.c_int32 * 4),
                ("tap_alpha", C.c_double * 4), ("pin_every_step", C.c_int32),
                ("clamp", C.c_int32)]


_libs = {}


def lib(parallel: bool = False):
    """The loaded oracle library: liborc.so, or with parallel=True the OpenMP
    build liborc_omp.so (same results, all host cores)."""
    L = _libs.get(parallel)
    if L is None:
        if parallel:
            os.environ.setdefault("OMP_NUM_THREADS", str(host_cores()))
            L = C.CDLL(build_parallel())
        else:
            L = C.CDLL(build())
        vp, i64, dbl = C.c_void_p, C.c_int64, C.c_double
        L.orc_create.restype = vp
        L.orc_create.argtypes = [vp, vp, vp]
        L.orc_destroy.argtypes = [vp]
        L.orc_sizes.argtypes = [vp, vp]
        L.orc_static_export.argtypes = [vp] * 6
        L.orc_nodes_export.argtypes = [vp] * 7
        L.orc_build_hints.argtypes = [vp, vp, vp, vp]
        L.orc_merged_export.argtypes = [vp] * 10
        L.orc_hr_steps.argtypes = [vp, C.c_int, vp, vp]
        L.orc_filter.argtypes = [vp] * 6
        L.orc_gift_band.argtypes = [vp, dbl, C.c_int, vp, vp]
        L.orc_gift.argtypes = [vp] * 6
        L.orc_init_signal.argtypes = [vp, C.c_uint64, vp, vp, vp]
        L.orc_run.argtypes = [vp, vp, C.c_uint64, vp, vp, vp]
        L.orc_hpwl.restype = dbl
        L.orc_hpwl.argtypes = [vp, vp, vp]
        L.orc_exp.restype = dbl
        L.orc_exp.argtypes = [dbl]
        L.orc_u01.restype = dbl
        L.orc_u01.argtypes = [C.c_uint64, C.c_uint64]
        L.orc_store.restype = dbl
        L.orc_store.argtypes = [dbl, C.c_int]
        L.orc_gauss_legendre.argtypes = [C.c_int, vp, vp]
        for f in ("orc_rho_eta", "orc_rho_sigma", "orc_rho_k"):
            getattr(L, f).restype = dbl
            getattr(L, f).argtypes = [vp, C.c_int]
        L.orc_rho_value.restype = dbl
        L.orc_rho_value.argtypes = [vp, C.c_int, dbl, dbl, dbl, dbl]
        L.orc_rho_integral.restype = dbl
        L.orc_rho_integral.argtypes = [vp, C.c_int, dbl, dbl, dbl, dbl, dbl, dbl]
        L.orc_macro_density.argtypes = [vp, C.c_int, C.c_int32, vp, vp, vp, vp, dbl, dbl, dbl,
                                         dbl, C.c_int32, C.c_int32, vp]
        _ = i64
        _libs[parallel] = L
    return L


def _p(a):
    return None if a is None else a.ctypes.data


def make_params(**kw) -> _Params:
    d = dict(DEFAULTS)
    d.update(kw)
    p = _Params()
    for k, v in d.items():
        if isinstance(v, (tuple, list)):
            arr = getattr(p, k)
            for j, x in enumerate(v):
                arr[j] = x
        else:
            setattr(p, k, v)
    return p


class _NetlistArrays:
    """Keeps contiguous copies alive while the C struct points at them."""

    def __init__(self, nl):
        self.net_ptr = np.ascontiguousarray(nl.net_ptr, np.int64)
        self.pin_cell = np.ascontiguousarray(nl.pin_cell, np.int32)
        self.pin_dx = None if nl.pin_dx is None else np.ascontiguousarray(nl.pin_dx, np.float32)
        self.pin_dy = None if nl.pin_dy is None else np.ascontiguousarray(nl.pin_dy, np.float32)
        self.cell_w = np.ascontiguousarray(nl.cell_w, np.float32)
        self.cell_h = np.ascontiguousarray(nl.cell_h, np.float32)
        self.cell_kind = np.ascontiguousarray(nl.cell_kind, np.uint8)
        self.fixed_x = np.ascontiguousarray(nl.fixed_x, np.float32)
        self.fixed_y = np.ascontiguousarray(nl.fixed_y, np.float32)
        s = _Netlist()
        s.num_cells = self.cell_w.shape[0]
        s.num_nets = self.net_ptr.shape[0] - 1
        s.num_pins = self.pin_cell.shape[0]
        s.net_ptr, s.pin_cell = _p(self.net_ptr), _p(self.pin_cell)
        s.pin_dx, s.pin_dy = _p(self.pin_dx), _p(self.pin_dy)
        s.cell_w, s.cell_h, s.cell_kind = _p(self.cell_w), _p(self.cell_h), _p(self.cell_kind)
        s.fixed_x, s.fixed_y = _p(self.fixed_x), _p(self.fixed_y)
        s.xl, s.yl, s.xh, s.yh = (float(v) for v in nl.region)
        self.struct = s


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"oracle {what} failed with code {code}")
        self.code = code


class Oracle:
    """One netlist's static graph plus the current augmented graph."""

    def __init__(self, nl, parallel=False, **params):
        self.nl = nl
        self._L = lib(parallel)
        self._arr = _NetlistArrays(nl)
        self.params = make_params(**params)
        err = C.c_int(0)
        self._g = self._L.orc_create(C.byref(self._arr.struct), C.byref(self.params), C.byref(err))
        if not self._g:
            raise OracleError(err.value, "create")
        s = np.zeros(16, np.int64)
        self._L.orc_sizes(self._g, s.ctypes.data)
        (self.C, self.Pm, self.S, self.Mm, self.NB, self.Nst, self.N, self.nnz_static) = \
            (int(v) for v in s[:8])
        self.hx, self.hy = int(s[9]), int(s[10])

    def __del__(self):
        if getattr(self, "_g", None):
            self._L.orc_destroy(self._g)
            self._g = None

    def sizes(self):
        s = np.zeros(16, np.int64)
        self._L.orc_sizes(self._g, s.ctypes.data)
        return s

    def static_csr(self):
        nnz = self.nnz_static
        rp = np.zeros(self.Nst + 1, np.int64)
        col = np.zeros(max(nnz, 1), np.int32)
        we = np.zeros(max(nnz, 1), np.float64)
        ws = np.zeros(max(nnz, 1), np.float64)
        bw = np.zeros(max(self.C, 1), np.float64)
        self._L.orc_static_export(self._g, rp.ctypes.data, col.ctypes.data, we.ctypes.data,
                                ws.ctypes.data, bw.ctypes.data)
        return dict(rp=rp, col=col[:nnz], w_exact=we[:nnz], w_store=ws[:nnz], base_w=bw[:self.C])

    def nodes(self):
        N = self.N
        nk = np.zeros(N, np.uint8)
        fx, fy, hw, hh = (np.zeros(N) for _ in range(4))
        pn = np.zeros(max(self.nl.num_pins, 1), np.int32)
        self._L.orc_nodes_export(self._g, nk.ctypes.data, fx.ctypes.data, fy.ctypes.data,
                               hw.ctypes.data, hh.ctypes.data, pn.ctypes.data)
        return dict(nkind=nk, fx=fx, fy=fy, hw=hw, hh=hh, pin_node=pn[:self.nl.num_pins])

    def build_hints(self, gx, gy, check=True):
        gx = np.ascontiguousarray(gx, np.float64)
        gy = np.ascontiguousarray(gy, np.float64)
        err = self._L.orc_build_hints(self._g, C.byref(self.params), gx.ctypes.data, gy.ctypes.data)
        if err and check:
            raise OracleError(err, "build_hints")
        return err

    def merged(self):
        s = self.sizes()
        nnz = int(s[8])
        N = self.N
        rp = np.zeros(N + 1, np.int64)
        col = np.zeros(max(nnz, 1), np.int32)
        w = np.zeros(max(nnz, 1))
        deg = np.zeros(N)
        lam = C.c_double(0)
        nb = max(self.NB, 1)
        Db, Cb, phi = np.zeros(nb), np.zeros(nb), np.zeros(nb)
        cb = np.zeros(max(self.C, 1), np.int32)
        self._L.orc_merged_export(self._g, rp.ctypes.data, col.ctypes.data, w.ctypes.data,
                                deg.ctypes.data, C.byref(lam), Db.ctypes.data, Cb.ctypes.data,
                                phi.ctypes.data, cb.ctypes.data)
        return dict(rp=rp, col=col[:nnz], w=w[:nnz], deg=deg, lam_up=lam.value,
                    Db=Db[:self.NB], Cb=Cb[:self.NB], phi=phi[:self.NB], cell_bin=cb[:self.C])

    def hr_steps(self, k, x):
        x = np.ascontiguousarray(x, np.float64)
        y = np.zeros(self.N)
        self._L.orc_hr_steps(self._g, int(k), x.ctypes.data, y.ctypes.data)
        return y

    def filter(self, gx, gy):
        gx = np.ascontiguousarray(gx, np.float64)
        gy = np.ascontiguousarray(gy, np.float64)
        ox, oy = np.zeros(self.N), np.zeros(self.N)
        self._L.orc_filter(self._g, C.byref(self.params), gx.ctypes.data, gy.ctypes.data,
                         ox.ctypes.data, oy.ctypes.data)
        return ox, oy

    def gift_band(self, sigma, k, x):
        x = np.ascontiguousarray(x, np.float64)
        y = np.zeros(self.N)
        err = self._L.orc_gift_band(self._g, float(sigma), int(k), x.ctypes.data, y.ctypes.data)
        if err:
            raise OracleError(err, "gift_band")
        return y

    def gift(self, gx, gy):
        gx = np.ascontiguousarray(gx, np.float64)
        gy = np.ascontiguousarray(gy, np.float64)
        ox, oy = np.zeros(self.N), np.zeros(self.N)
        err = self._L.orc_gift(self._g, C.byref(self.params), gx.ctypes.data, gy.ctypes.data,
                             ox.ctypes.data, oy.ctypes.data)
        if err:
            raise OracleError(err, "gift")
        return ox, oy

    def init_signal(self, seed, xy0=None):
        gx, gy = np.zeros(self.N), np.zeros(self.N)
        x0 = None if xy0 is None else np.ascontiguousarray(xy0, np.float32)
        self._L.orc_init_signal(self._g, C.c_uint64(seed), _p(x0), gx.ctypes.data, gy.ctypes.data)
        return gx, gy

    def run(self, seed, xy0=None, check=True):
        gx, gy = np.zeros(self.N), np.zeros(self.N)
        x0 = None if xy0 is None else np.ascontiguousarray(xy0, np.float32)
        err = self._L.orc_run(self._g, C.byref(self.params), C.c_uint64(seed), _p(x0),
                            gx.ctypes.data, gy.ctypes.data)
        if err and check:
            raise OracleError(err, "run")
        return gx, gy


def hpwl(nl, cx, cy, parallel=False) -> float:
    a = _NetlistArrays(nl)
    cx = np.ascontiguousarray(cx, np.float64)
    cy = np.ascontiguousarray(cy, np.float64)
    return lib(parallel).orc_hpwl(C.byref(a.struct), cx.ctypes.data, cy.ctypes.data)


def exp(x: float) -> float:
    return lib().orc_exp(float(x))


def u01(seed: int, ctr: int) -> float:
    return lib().orc_u01(C.c_uint64(seed), C.c_uint64(ctr))


def store(w: float, dtype: int) -> float:
    return lib().orc_store(float(w), int(dtype))


# ----------------------------------------------- Sec. VI charge schedules
RHO_GAUSS, RHO_EXP, RHO_LINEAR, RHO_SIGMOID = 0, 1, 2, 3


class RhoParams(C.Structure):
    _fields_ = [("model", C.c_int32), ("T", C.c_int32), ("r0", C.c_double), ("r1", C.c_double),
                ("beta_min", C.c_double), ("beta_max", C.c_double), ("alpha0", C.c_double),
                ("alpha1", C.c_double), ("sigma_factor", C.c_double), ("k_factor", C.c_double),
                ("panels", C.c_int32), ("nodes", C.c_int32)]


# Readings (the paper gives T = 300 for its figure and no other value).
RHO_DEFAULTS = dict(model=RHO_GAUSS, T=300, r0=0.05, r1=0.9, beta_min=0.25, beta_max=1.5,
                    alpha0=0.3, alpha1=0.7, sigma_factor=0.002, k_factor=0.5, panels=4, nodes=8)


def rho_params(**kw) -> RhoParams:
    d = dict(RHO_DEFAULTS)
    d.update(kw)
    p = RhoParams()
    for k, v in d.items():
        setattr(p, k, v)
    return p


def gauss_legendre(n):
    x, w = np.zeros(n), np.zeros(n)
    lib().orc_gauss_legendre(int(n), x.ctypes.data, w.ctypes.data)
    return x, w


def rho_eta(rp, t):
    return lib().orc_rho_eta(C.byref(rp), int(t))


def rho_sigma(rp, t):
    return lib().orc_rho_sigma(C.byref(rp), int(t))


def rho_k(rp, t):
    return lib().orc_rho_k(C.byref(rp), int(t))


def rho_value(rp, t, dx, dy, w, h):
    return lib().orc_rho_value(C.byref(rp), int(t), dx, dy, w, h)


def rho_integral(rp, t, w, h, ax, bx, ay, by):
    return lib().orc_rho_integral(C.byref(rp), int(t), w, h, ax, bx, ay, by)


def macro_density(rp, t, mx, my, mw, mh, region, nbx, nby):
    """Per-bin integral of the macros' scheduled charge (area units)."""
    a = [np.ascontiguousarray(v, np.float64) for v in (mx, my, mw, mh)]
    out = np.zeros(nbx * nby)
    xl, yl, xh, yh = region
    lib().orc_macro_density(C.byref(rp), int(t), len(a[0]), *(v.ctypes.data for v in a),
                            xl, yl, xh, yh, int(nbx), int(nby), out.ctypes.data)
    return out
