"""Python binding of libpl, the GB300 area-hint refinement initializer.

Argument marshalling only: every step of the path runs in the CUDA library
(libpl.so, built in-tree by build.py).  PyTorch provides device memory and
streams.  Functions keep the C names (pl_build_graph, pl_filter_init,
pl_hpwl, ...); see include/pl.h for the contract of each call.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpl.so")

PL_OK, PL_ERR_INVALID_ARG, PL_ERR_CUDA, PL_ERR_WORKSPACE, PL_ERR_OOM, PL_ERR_SPECTRUM, \
    PL_ERR_NONFINITE, PL_ERR_TIMEOUT, PL_ERR_UNSUPPORTED = range(9)
PL_W_FP32, PL_W_BF16 = 1, 2


class PlError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libpl error {code}: {msg}")
        self.code = code


class PlNetlist(C.Structure):
    _fields_ = [("num_cells", C.c_int32), ("num_nets", C.c_int32), ("num_pins", C.c_int64),
                ("net_ptr", C.c_void_p), ("pin_cell", C.c_void_p),
                ("pin_dx", C.c_void_p), ("pin_dy", C.c_void_p),
                ("cell_w", C.c_void_p), ("cell_h", C.c_void_p), ("cell_kind", C.c_void_p),
                ("fixed_x", C.c_void_p), ("fixed_y", C.c_void_p),
                ("xl", C.c_double), ("yl", C.c_double), ("xh", C.c_double), ("yh", C.c_double)]


class PlParams(C.Structure):
    _fields_ = [("clique_max", C.c_int32), ("wdtype", C.c_int32),
                ("gift_enable", C.c_int32), ("gift_center", C.c_int32),
                ("gift_k", C.c_int32 * 3), ("gift_sigma", C.c_double * 3),
                ("gift_alpha", C.c_double * 3), ("t_hint", C.c_int32),
                ("nbx", C.c_int32), ("nby", C.c_int32),
                ("gamma", C.c_double), ("det_ratio", C.c_double), ("capacity", C.c_double),
                ("mu", C.c_double), ("ntaps", C.c_int32), ("tap_k", C.c_int32 * 4),
                ("tap_alpha", C.c_double * 4), ("pin_every_step", C.c_int32),
                ("clamp", C.c_int32)]

    def as_dict(self) -> dict:
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = tuple(v) if hasattr(v, "__len__") else v
        return out


_lib = None


def lib():
    """The loaded libpl.so.  Raises if it has not been built: there is no
    fallback implementation."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_2511_10073_gb300.build.build() (nvcc, sm_103a)")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, u64, dbl, sz = (C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double,
                                      C.c_size_t)
        sigs = {
            "pl_params_default": (None, [vp]),
            "pl_workspace_size": (sz, [vp, vp]),
            "pl_build_graph": (C.c_int, [vp, vp, vp, vp, sz, vp, vp]),
            "pl_graph_info": (C.c_int, [vp, vp]),
            "pl_build_hints": (C.c_int, [vp, vp, vp, vp]),
            "pl_filter_apply": (C.c_int, [vp, vp, vp, vp, vp]),
            "pl_gift": (C.c_int, [vp, vp, vp, vp, vp]),
            "pl_init_signal": (C.c_int, [vp, u64, vp, vp, vp]),
            "pl_filter_init": (C.c_int, [vp, vp, u64, vp, vp, vp]),
            "pl_hpwl_workspace_size": (sz, [i32]),
            "pl_hpwl": (C.c_int, [vp, vp, vp, vp, sz, vp]),
            "pl_hpwl_noalloc": (C.c_int, [vp, vp, vp, vp]),
            "pl_graph_export_static": (C.c_int, [vp, vp, vp, vp, vp]),
            "pl_graph_export": (C.c_int, [vp] * 10),
            "pl_graph_destroy": (None, [vp]),
            "pl_last_error": (C.c_char_p, []),
            "pl_filter_init_batch": (C.c_int, [i32, vp, vp, vp, vp, i32, vp, vp, vp, sz]),
            "pl_batch_opts_default": (None, [vp]),
            "pl_batch_workspace_size": (sz, [i32, vp]),
            "pl_batch_autotune": (C.c_int, [i32, vp, vp, vp, vp, i32, vp, vp, sz, vp, vp]),
            "pl_rho_params_default": (None, [vp]),
            "pl_macro_density": (C.c_int, [vp, i32, i32, vp, vp, vp, vp, dbl, dbl, dbl, dbl,
                                           i32, i32, vp, vp]),
            "pl_learned_apply": (C.c_int, [vp, vp, vp, i32, vp, vp, vp]),
            "pl_filter_init_learned": (C.c_int, [vp, vp, vp, u64, vp, vp, vp, vp]),
            "pl_learned_forward": (C.c_int, [vp, vp, i64, vp, vp]),
            "pl_learned_wait_check": (C.c_int, [i64, vp, sz, vp]),
            "pl_learned_collect": (C.c_int, [vp, vp, vp, i32, vp, vp, i64, vp, vp]),
            "pl_train_opts_default": (None, [vp]),
            "pl_learned_train_ws": (sz, [i64]),
            "pl_learned_train": (C.c_int, [vp, i64, vp, vp, vp, sz, vp, vp]),
            "pl_learned_loss": (C.c_int, [vp, i64, vp, vp, sz, vp, vp, vp]),
            "pl_prof_enable": (None, [C.c_int]),
            "pl_prof_read": (C.c_int, [vp]),
        }
        for name, (res, args) in sigs.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _ = (i64, dbl)
        _lib = L
    return _lib


def _check(code: int):
    if code != PL_OK:
        raise PlError(code, lib().pl_last_error().decode())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def params(**kw) -> PlParams:
    """pl_params_default() with the given fields replaced."""
    p = PlParams()
    lib().pl_params_default(C.byref(p))
    for k, v in kw.items():
        if isinstance(v, (tuple, list)):
            arr = getattr(p, k)
            for j, x in enumerate(v):
                arr[j] = x
        else:
            setattr(p, k, v)
    return p


class DeviceNetlist:
    """Netlist arrays resident on the device plus the C struct that points at
    them (kept alive together)."""

    def __init__(self, nl, device="cuda"):
        import torch
        t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a)).to(device=device, dtype=dt)
        self.net_ptr = t(nl.net_ptr, torch.int64)
        self.pin_cell = t(nl.pin_cell, torch.int32)
        self.pin_dx = None if nl.pin_dx is None else t(nl.pin_dx, torch.float32)
        self.pin_dy = None if nl.pin_dy is None else t(nl.pin_dy, torch.float32)
        self.cell_w = t(nl.cell_w, torch.float32)
        self.cell_h = t(nl.cell_h, torch.float32)
        self.cell_kind = t(nl.cell_kind, torch.uint8)
        self.fixed_x = t(nl.fixed_x, torch.float32)
        self.fixed_y = t(nl.fixed_y, torch.float32)
        self.region = tuple(float(v) for v in nl.region)
        s = PlNetlist()
        s.num_cells = self.cell_w.numel()
        s.num_nets = self.net_ptr.numel() - 1
        s.num_pins = self.pin_cell.numel()
        s.net_ptr, s.pin_cell = self.net_ptr.data_ptr(), self.pin_cell.data_ptr() if s.num_pins else 0
        s.pin_dx = self.pin_dx.data_ptr() if self.pin_dx is not None and s.num_pins else None
        s.pin_dy = self.pin_dy.data_ptr() if self.pin_dy is not None and s.num_pins else None
        for f in ("cell_w", "cell_h", "cell_kind", "fixed_x", "fixed_y"):
            setattr(s, f, getattr(self, f).data_ptr() if s.num_cells else None)
        s.xl, s.yl, s.xh, s.yh = self.region
        self.struct = s
        self.num_cells, self.num_nets = s.num_cells, s.num_nets


class Graph:
    """A pl_graph handle and the workspace tensor that holds its device
    memory (the library allocates none)."""

    def __init__(self, handle: C.c_void_p, netlist: DeviceNetlist, ws=None):
        self._h = handle
        self.netlist = netlist
        self.ws = ws

    def __del__(self):
        self.destroy()

    def destroy(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().pl_graph_destroy(self._h)
            self._h = C.c_void_p(None)

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        out = np.zeros(16, np.int64)
        _check(lib().pl_graph_info(self._h, out.ctypes.data))
        keys = ["num_cells", "macro_pins", "stars", "macros", "bins", "static_nodes", "N",
                "static_nnz", "nnz", "hx", "hy", "hub_rows", "movable", "ws_peak", "ws_bytes",
                "ws_static"]
        return {k: int(out[i]) for i, k in enumerate(keys)}

    def export_static(self) -> dict:
        inf = self.info()
        n, nnz, c = inf["static_nodes"], inf["static_nnz"], inf["num_cells"]
        rp = np.zeros(n + 1, np.int64)
        col = np.zeros(max(nnz, 1), np.int32)
        w = np.zeros(max(nnz, 1))
        bw = np.zeros(max(c, 1))
        _check(lib().pl_graph_export_static(self._h, rp.ctypes.data, col.ctypes.data,
                                            w.ctypes.data, bw.ctypes.data))
        return dict(rp=rp, col=col[:nnz], w=w[:nnz], base_w=bw[:c])

    def export(self) -> dict:
        inf = self.info()
        N, nnz, nb, c = inf["N"], inf["nnz"], inf["bins"], inf["num_cells"]
        rp = np.zeros(N + 1, np.int64)
        col = np.zeros(max(nnz, 1), np.int32)
        w = np.zeros(max(nnz, 1))
        deg = np.zeros(N)
        lam = C.c_double(0)
        Db, Cb, phi = np.zeros(nb), np.zeros(nb), np.zeros(nb)
        cb = np.zeros(max(c, 1), np.int32)
        _check(lib().pl_graph_export(self._h, rp.ctypes.data, col.ctypes.data, w.ctypes.data,
                                     deg.ctypes.data, C.byref(lam), Db.ctypes.data,
                                     Cb.ctypes.data, phi.ctypes.data, cb.ctypes.data))
        return dict(rp=rp, col=col[:nnz], w=w[:nnz], deg=deg, lam_up=lam.value, Db=Db, Cb=Cb,
                    phi=phi, cell_bin=cb[:c])


def pl_workspace_size(dnl: DeviceNetlist, prm: PlParams) -> int:
    return int(lib().pl_workspace_size(C.byref(dnl.struct), C.byref(prm)))


def workspace(nbytes: int, device="cuda"):
    """A device workspace (a torch allocation, 256-byte aligned)."""
    import torch
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def pl_build_graph(dnl: DeviceNetlist, prm: PlParams, xy_nodes=None, stream=None,
                   graph: Graph | None = None, ws=None) -> Graph:
    """Builds (or, given `graph`, rebuilds in place) a graph in the device
    workspace `ws`: by default the graph's current one when large enough,
    else a new torch allocation of pl_workspace_size bytes."""
    if ws is None:
        need = pl_workspace_size(dnl, prm)
        if graph is not None and graph.ws is not None and graph.ws.numel() >= need:
            ws = graph.ws
        else:
            ws = workspace(need, dnl.cell_w.device)
    h = graph.handle if graph is not None else C.c_void_p(None)
    _check(lib().pl_build_graph(C.byref(dnl.struct), C.byref(prm), _ptr(xy_nodes), _ptr(ws),
                                C.c_size_t(ws.numel() * ws.element_size()), _stream(stream),
                                C.byref(h)))
    if graph is not None:
        graph._h = h
        graph.netlist = dnl
        graph.ws = ws
        return graph
    return Graph(h, dnl, ws)


def pl_build_hints(g: Graph, prm: PlParams, xy_nodes, stream=None):
    _check(lib().pl_build_hints(g.handle, C.byref(prm), _ptr(xy_nodes), _stream(stream)))


def pl_filter_apply(g: Graph, prm: PlParams, xy_in, xy_out, stream=None):
    _check(lib().pl_filter_apply(g.handle, C.byref(prm), _ptr(xy_in), _ptr(xy_out),
                                 _stream(stream)))


def pl_gift(g: Graph, prm: PlParams, xy_in, xy_out, stream=None):
    _check(lib().pl_gift(g.handle, C.byref(prm), _ptr(xy_in), _ptr(xy_out), _stream(stream)))


def pl_init_signal(g: Graph, seed: int, xy0_cells, xy_nodes, stream=None):
    _check(lib().pl_init_signal(g.handle, C.c_uint64(seed), _ptr(xy0_cells), _ptr(xy_nodes),
                                _stream(stream)))


def pl_filter_init(g: Graph, prm: PlParams, seed: int, xy0_cells, xy_out_cells, stream=None):
    _check(lib().pl_filter_init(g.handle, C.byref(prm), C.c_uint64(seed), _ptr(xy0_cells),
                                _ptr(xy_out_cells), _stream(stream)))


class PlBatchOpts(C.Structure):
    _fields_ = [("union_products", C.c_int32), ("streams", C.c_int32),
                ("rows_ctas_per_sm", C.c_int32)]


def batch_opts(**kw) -> PlBatchOpts:
    o = PlBatchOpts()
    lib().pl_batch_opts_default(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def batch_workspace(n: int, prm: PlParams, device="cuda"):
    import torch
    nb = int(lib().pl_batch_workspace_size(int(n), C.byref(prm)))
    return torch.empty(max(nb, 256), dtype=torch.uint8, device=device)


def _batch_args(graphs, seeds, outs, streams):
    n = len(graphs)
    gh = (C.c_void_p * n)(*[g.handle.value for g in graphs])
    sd = (C.c_uint64 * n)(*[int(x) for x in seeds])
    op = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
    sp = (C.c_void_p * len(streams))(*[s.cuda_stream for s in streams])
    return n, gh, sd, op, sp


def pl_filter_init_batch(graphs, prm: PlParams, seeds, outs, streams, opts: PlBatchOpts | None = None,
                         ws=None):
    """The initializer of every design of a batch (see include/pl.h):
    outs[i] is a device tensor of graphs[i]'s num_cells pairs; streams are
    torch CUDA streams (one worker thread each).  The union form (the
    default) takes a device workspace (allocated here when ws is None)."""
    n, gh, sd, op, sp = _batch_args(graphs, seeds, outs, streams)
    if opts is None:
        opts = batch_opts()
    if ws is None and opts.union_products:
        ws = batch_workspace(n, prm, outs[0].device)
    nb = 0 if ws is None else ws.numel()
    _check(lib().pl_filter_init_batch(n, gh, C.byref(prm), sd, op, len(streams), sp,
                                      C.byref(opts), _ptr(ws), C.c_size_t(nb)))


def pl_batch_autotune(graphs, prm: PlParams, seeds, outs, streams, ws=None):
    """Runs every candidate of the batch autotuner; returns (best options,
    best ms)."""
    n, gh, sd, op, sp = _batch_args(graphs, seeds, outs, streams)
    if ws is None:
        ws = batch_workspace(n, prm, outs[0].device)
    best = PlBatchOpts()
    ms = C.c_double(0)
    _check(lib().pl_batch_autotune(n, gh, C.byref(prm), sd, op, len(streams), sp, _ptr(ws),
                                   C.c_size_t(ws.numel()), C.byref(best), C.byref(ms)))
    return best, float(ms.value)


def pl_hpwl_workspace_size(num_nets: int) -> int:
    return int(lib().pl_hpwl_workspace_size(int(num_nets)))


def pl_hpwl(dnl: DeviceNetlist, xy_cells, out, ws, stream=None):
    _check(lib().pl_hpwl(C.byref(dnl.struct), _ptr(xy_cells), _ptr(out), _ptr(ws),
                         C.c_size_t(ws.numel() * ws.element_size()), _stream(stream)))


def pl_hpwl_noalloc(dnl: DeviceNetlist, xy_cells, out, stream=None):
    """HPWL into `out` (device double) with the library's fixed scratch: no
    workspace, no allocation (see include/pl.h)."""
    _check(lib().pl_hpwl_noalloc(C.byref(dnl.struct), _ptr(xy_cells), _ptr(out), _stream(stream)))


def hpwl_workspace(num_nets: int, device="cuda"):
    """A device workspace for pl_hpwl (256-byte aligned torch allocation)."""
    import torch
    return torch.empty(pl_hpwl_workspace_size(num_nets), dtype=torch.uint8, device=device)


def pl_prof_enable(on: bool):
    lib().pl_prof_enable(1 if on else 0)


def pl_prof_read() -> dict:
    out = np.zeros(8)
    _check(lib().pl_prof_read(out.ctypes.data))
    return dict(launches=int(out[0]), hr_launches=int(out[1]), hr_ms=float(out[2]),
                hr_bytes=float(out[3]), gift_launches=int(out[4]), gift_ms=float(out[5]),
                gift_bytes=float(out[6]))


# ------------------------------------------- Sec. VI macro charge schedules
PL_RHO_GAUSS, PL_RHO_EXP, PL_RHO_LINEAR, PL_RHO_SIGMOID = range(4)


class PlRhoParams(C.Structure):
    _fields_ = [("model", C.c_int32), ("T", C.c_int32), ("r0", C.c_double), ("r1", C.c_double),
                ("beta_min", C.c_double), ("beta_max", C.c_double), ("alpha0", C.c_double),
                ("alpha1", C.c_double), ("sigma_factor", C.c_double), ("k_factor", C.c_double),
                ("panels", C.c_int32), ("nodes", C.c_int32)]


def rho_params(**kw) -> PlRhoParams:
    """pl_rho_params_default() with the given fields replaced."""
    p = PlRhoParams()
    lib().pl_rho_params_default(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def pl_macro_density(rp: PlRhoParams, t: int, mx, my, mw, mh, region, nbx: int, nby: int, out,
                     stream=None):
    """Per-bin integral (device doubles `out`) of the macros' charge at
    iteration t; mx..mh are device float tensors."""
    xl, yl, xh, yh = (float(v) for v in region)
    _check(lib().pl_macro_density(C.byref(rp), int(t), int(mx.numel()), _ptr(mx), _ptr(my),
                                  _ptr(mw), _ptr(mh), xl, yl, xh, yh, int(nbx), int(nby),
                                  _ptr(out), _stream(stream)))


# ------------------------------------------- the learned refinement filter
LEARNED_NF, LEARNED_HID, LEARNED_NOUT = 16, 64, 4
LW_MU, LW_ISD, LW_THETA, LW_W1, LW_B1, LW_W2, LW_B2, LEARNED_SIZE = 0, 16, 32, 35, 1059, 1123, 1379, 1383
LEARNED_REC = 24


class PlLearned(C.Structure):
    _fields_ = [("k", C.c_int32 * 3), ("w", C.c_void_p)]


class PlTrainOpts(C.Structure):
    _fields_ = [("epochs", C.c_int32), ("batch_tiles", C.c_int32), ("lr", C.c_double),
                ("lr_min", C.c_double), ("beta1", C.c_double), ("beta2", C.c_double),
                ("eps", C.c_double), ("seed", C.c_uint64), ("fit_norm", C.c_int32),
                ("fit_taps", C.c_int32)]


class LearnedModel:
    """Tap powers k = (k0, k1, k2) and the device parameter vector `w`
    (PL_LEARNED_SIZE floats), with the C struct that points at them."""

    def __init__(self, k, w):
        self.k = tuple(int(x) for x in k)
        self.w = w
        self.struct = PlLearned((C.c_int32 * 3)(*self.k), C.c_void_p(w.data_ptr()))

    def host(self) -> dict:
        return {"k": list(self.k), "w": [float(x) for x in self.w.detach().cpu().numpy()]}

    @staticmethod
    def from_host(d: dict, device="cuda") -> "LearnedModel":
        import torch
        return LearnedModel(d["k"], torch.tensor(d["w"], dtype=torch.float32, device=device))


def learned_init(k, seed: int, device="cuda") -> LearnedModel:
    """A fresh parameter vector: W1 ~ N(0, 1/16) (He-like for 16 inputs) from
    numpy's PCG64(seed), every other weight zero, isd 1 (normalisation and
    taps are fitted by pl_learned_train)."""
    import torch
    w = np.zeros(LEARNED_SIZE, np.float32)
    w[LW_ISD:LW_ISD + LEARNED_NF] = 1.0
    w[LW_THETA + 2] = 1.0
    rng = np.random.Generator(np.random.PCG64(seed))
    w[LW_W1:LW_B1] = rng.normal(0.0, 0.25, LEARNED_HID * LEARNED_NF)
    return LearnedModel(k, torch.tensor(w, device=device))


def train_opts(**kw) -> PlTrainOpts:
    o = PlTrainOpts()
    lib().pl_train_opts_default(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def pl_learned_apply(g: Graph, prm: PlParams, m: LearnedModel, rnd: int, xy_in, xy_out,
                     stream=None):
    _check(lib().pl_learned_apply(g.handle, C.byref(prm), C.byref(m.struct), int(rnd),
                                  _ptr(xy_in), _ptr(xy_out), _stream(stream)))


def pl_filter_init_learned(g: Graph, prm: PlParams, m: LearnedModel | None, seed: int, xy0_cells,
                           xy_out_cells, stream=None) -> int:
    """The whole initializer with the learned filter; returns the number of
    rounds that fell back to the plain filter."""
    nf = C.c_int32(0)
    _check(lib().pl_filter_init_learned(g.handle, C.byref(prm),
                                        None if m is None else C.byref(m.struct), C.c_uint64(seed),
                                        _ptr(xy0_cells), _ptr(xy_out_cells), C.byref(nf),
                                        _stream(stream)))
    return int(nf.value)


def pl_learned_wait_check(cycles: int, ws=None, stream=None) -> int:
    """Runs the bounded-wait check; returns its status code (PL_ERR_TIMEOUT
    when the wait gave up, as it should)."""
    import torch
    if ws is None:
        ws = torch.empty(8192, dtype=torch.uint8, device="cuda")
    code = lib().pl_learned_wait_check(int(cycles), _ptr(ws), C.c_size_t(ws.numel()), _stream(stream))
    if code not in (PL_OK, PL_ERR_TIMEOUT):
        _check(code)
    return int(code)


def pl_learned_forward(w, feat, out, stream=None):
    _check(lib().pl_learned_forward(_ptr(w), _ptr(feat), int(feat.shape[0]), _ptr(out),
                                    _stream(stream)))


def pl_learned_collect(g: Graph, prm: PlParams, k, rnd: int, xy_in, rec, stream=None) -> int:
    """Writes this round's records into the device float tensor `rec`
    (rows of LEARNED_REC floats) and returns their count; with rec None,
    only returns the count."""
    kk = (C.c_int32 * 3)(*[int(x) for x in k])
    cnt = C.c_int64(0)
    cap = 0 if rec is None else rec.numel() // LEARNED_REC
    code = lib().pl_learned_collect(g.handle, C.byref(prm), kk, int(rnd), _ptr(xy_in), _ptr(rec),
                                    cap, C.byref(cnt), _stream(stream))
    if rec is None and code == PL_ERR_WORKSPACE:
        return int(cnt.value)  # the count asked for
    _check(code)
    return int(cnt.value)


def learned_train_workspace(nrec: int, device="cuda"):
    import torch
    return torch.empty(max(int(lib().pl_learned_train_ws(int(nrec))), 256), dtype=torch.uint8,
                       device=device)


def pl_learned_train(rec, nrec: int, m: LearnedModel, opts: PlTrainOpts, ws=None,
                     stream=None) -> list:
    """Trains m.w in place on the first nrec rows of `rec`; returns the
    per-epoch mean minibatch loss."""
    if ws is None:
        ws = learned_train_workspace(nrec, rec.device)
    loss = np.zeros(max(opts.epochs, 1))
    _check(lib().pl_learned_train(_ptr(rec), int(nrec), _ptr(m.w), C.byref(opts), _ptr(ws),
                                  C.c_size_t(ws.numel()), loss.ctypes.data, _stream(stream)))
    return [float(x) for x in loss[:opts.epochs]]


def pl_learned_loss(rec, nrec: int, w, grad=None, ws=None, stream=None) -> float:
    if ws is None:
        ws = learned_train_workspace(nrec, rec.device)
    loss = C.c_double(0)
    _check(lib().pl_learned_loss(_ptr(rec), int(nrec), _ptr(w), _ptr(ws), C.c_size_t(ws.numel()),
                                 C.byref(loss), _ptr(grad), _stream(stream)))
    return float(loss.value)
