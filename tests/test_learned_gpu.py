"""GPU parity of the learned refinement filter against the FP64 oracle
(oracle/learned.py), through the C ABI:
  * the tensor-core MLP (pl_learned_forward): bit-exact where every sum is
    exact in FP32 (small dyadic inputs and weights), and within the
    arithmetic's tolerance on random inputs, over several persistent tiles and
    a ragged last tile;
  * training records (pl_learned_collect): taps, features and targets of one
    round against the oracle's from the same FP32 input;
  * one learned round (pl_learned_apply): coordinates within 1e-4 of the die;
  * the loss and its gradient (pl_learned_loss), one Adam step and the fitted
    normalisation and taps (pl_learned_train) on seeded records;
  * the whole initializer with the learned filter: no model gives the plain
    initializer's bits; a model whose output is not finite falls back to the
    plain filter in every round.
Every oracle input is seeded or the oracle's own output rounded to FP32.
"""
import numpy as np
import pytest

import oracle
from oracle import learned as L
from paper_2511_10073_gb300 import netgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def pl():
    import paper_2511_10073_gb300 as m
    return m


def dev(a, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def random_model(seed, w1=0.3, w2=0.1, theta=(0.3, -0.6, 1.3)):
    rng = np.random.default_rng(seed)
    p = {"mu": rng.normal(0, 0.3, L.NF), "isd": rng.uniform(0.5, 2.0, L.NF),
         "theta": np.array(theta), "W1": rng.normal(0, w1, (L.HID, L.NF)),
         "b1": rng.normal(0, 0.1, L.HID), "W2": rng.normal(0, w2, (L.NOUT, L.HID)),
         "b2": rng.normal(0, 0.05, L.NOUT)}
    w = L.pack(p).astype(np.float32)          # the device holds FP32 weights
    return w, L.unpack(w.astype(np.float64))  # the oracle reads the same values


# ------------------------------------------------------- the MLP alone
def test_forward_exact_on_dyadic_inputs():
    """Inputs in {-4..4}, W1 in {-1/4, 0, 1/4}, b1 in quarters, W2 in
    {-1/8, 0, 1/8}: every product and sum is exact in FP32 and every hidden
    value exact in BF16, so the tensor cores must give the oracle's bits.  A
    transposed operand, a wrong core-matrix offset or a lost K slab fails."""
    rng = np.random.default_rng(11)
    n = 128 * 7 + 45
    f = rng.integers(-4, 5, (n, L.NF)).astype(np.float64)
    p = {"mu": np.zeros(L.NF), "isd": np.ones(L.NF), "theta": np.zeros(3),
         "W1": rng.integers(-1, 2, (L.HID, L.NF)) / 4.0, "b1": rng.integers(-4, 5, L.HID) / 4.0,
         "W2": rng.integers(-1, 2, (L.NOUT, L.HID)) / 8.0, "b2": rng.integers(-4, 5, L.NOUT) / 8.0}
    w = L.pack(p).astype(np.float32)
    out = torch.full((n, 4), float("nan"), device="cuda")
    pl().pl_learned_forward(dev(w), dev(f), out)
    torch.cuda.synchronize()
    _, _, want = L.mlp_forward(L.normalise(f, p["mu"], p["isd"]), p)
    assert np.array_equal(out.cpu().numpy().astype(np.float64), want)


@pytest.mark.parametrize("n", [1, 128 * 5 + 37, 200_003])
def test_forward_matches_oracle(n):
    """Random weights and features.  FP32 accumulation in another order and
    FP32 normalisation round a value to the other side of a BF16 tie now and
    then, which moves that output by about 2^-8 of one hidden term; all other
    outputs agree to 1e-5 of the sum of their terms' magnitudes."""
    w, p = random_model(5)
    rng = np.random.default_rng(n)
    f = rng.normal(0, 1.5, (n, L.NF)).astype(np.float32).astype(np.float64)
    out = torch.full((n, 4), float("nan"), device="cuda")
    pl().pl_learned_forward(dev(w), dev(f), out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    _, hb, want = L.mlp_forward(L.normalise(f, p["mu"], p["isd"]), p)
    terms = np.abs(hb) @ np.abs(L.bf16(p["W2"])).T + np.abs(p["b2"])
    err = np.abs(got - want)
    assert np.isfinite(got).all()
    tight = err <= 1e-5 * terms + 1e-30
    assert tight.mean() >= 0.98, tight.mean()
    assert (err <= 2e-2 * terms + 1e-30).all(), float((err / terms).max())


# --------------------------------------------- one round on a real graph
class Round:
    """A netlist on both sides with the area hints built at the oracle's
    GiFt output rounded to FP32 (the round's input on both sides)."""

    def __init__(self, cfg, seed, **kw):
        m = pl()
        self.nl = netgen.make_netlist(cfg, seed)
        self.kw = kw
        self.prm = m.params(**kw)
        self.dnl = m.DeviceNetlist(self.nl)
        self.g = m.pl_build_graph(self.dnl, self.prm)
        self.N = self.g.info()["N"]
        self.o = oracle.Oracle(self.nl, **kw)
        ox, oy = self.o.init_signal(seed)
        a0 = np.stack([ox, oy], 1).astype(np.float32).astype(np.float64)
        gx, gy = self.o.gift(a0[:, 0], a0[:, 1])
        a = np.stack([gx, gy], 1).astype(np.float32)
        self.ax, self.ay = a[:, 0].astype(np.float64), a[:, 1].astype(np.float64)
        self.xy = dev(a.reshape(-1))
        m.pl_build_hints(self.g, self.prm, self.xy)
        self.o.build_hints(self.ax, self.ay)
        xl, yl, xh, yh = self.nl.region
        self.die = xh - xl
        self.tol_bins = np.array([1e-4 * (xh - xl) / ((xh - xl) / self.prm.nbx),
                                  1e-4 * (xh - xl) / ((yh - yl) / self.prm.nby)])

    def oracle_target(self):
        """The filter output that the relaxation maps to the plain round's
        result (the records' target)."""
        tx, ty = self.o.filter(self.ax, self.ay)
        return L.effective_target(np.stack([tx, ty], 1), np.stack([self.ax, self.ay], 1),
                                  self.o.params.gamma)


@pytest.mark.parametrize("cfg,seed,kw,k,rnd", [
    ("tiny", 2, dict(nbx=16, nby=16), (0, 2, 4), 1),
    ("tiny", 3, dict(nbx=16, nby=16, wdtype=2, ntaps=3, tap_k=(2, 4, 8, 0),
                     tap_alpha=(1 / 3, 1 / 3, 1 / 3, 0)), (1, 2, 3), 0),
    ("small", 1, dict(nbx=8, nby=8, det_ratio=0.4, pin_every_step=1), (0, 1, 2), 2)])
def test_collect_matches_oracle(cfg, seed, kw, k, rnd):
    m = pl()
    s = Round(cfg, seed, **kw)
    n = m.pl_learned_collect(s.g, s.prm, k, rnd, s.xy, None)
    rec = torch.full(((n + 3) * m.LEARNED_REC,), float("nan"), device="cuda")
    assert m.pl_learned_collect(s.g, s.prm, k, rnd, s.xy, rec) == n
    torch.cuda.synchronize()
    R = rec.view(-1, m.LEARNED_REC).double().cpu().numpy()
    assert np.isnan(R[n:]).all()  # nothing past the count
    R = R[:n]
    r = L.round_inputs(s.o, s.ax, s.ay, k, rnd)
    fr = r["free"]
    assert n == int(fr.sum())
    T = L.bins(s.oracle_target(), r["c"], r["s"])[fr]
    tol = s.tol_bins
    for j, G in enumerate((r["G0"], r["G1"], r["G2"])):
        assert (np.abs(R[:, 16 + 2 * j:18 + 2 * j] - G[fr]) <= tol).all(), j
    # the round result within 1e-4 of the die, divided by gamma; FP32 rounding
    # of (g' - (1 - gamma) g) / gamma at the coordinates' scale
    assert (np.abs(R[:, 22:24] - T) <= tol / s.prm.gamma + 1e-5 * (1 + np.abs(T))).all()
    f = r["f"][fr]
    assert (np.abs(R[:, 0:4] - f[:, 0:4]) <= 2 * np.r_[tol, tol]).all()
    assert (np.abs(R[:, 4:7] - f[:, 4:7]) <= 1e-5 * np.abs(f[:, 4:7]) + 1e-7).all()
    assert (np.abs(R[:, 7] - f[:, 7]) <= 1e-6 * np.abs(f[:, 7])).all()
    assert np.array_equal(R[:, 8:10], f[:, 8:10])
    assert (np.abs(R[:, 10] - f[:, 10]) <= 1e-6 * f[:, 10]).all()
    assert np.array_equal(R[:, 11], f[:, 11].astype(np.float32).astype(np.float64))
    assert np.all(R[:, 12:16] == 0)


@pytest.mark.parametrize("cfg,seed,kw,k,rnd", [
    ("tiny", 2, dict(nbx=16, nby=16), (0, 2, 4), 1),
    ("tiny", 5, dict(nbx=16, nby=16, wdtype=2, gamma=0.7), (0, 1, 2), 0),
    ("medium", 1, dict(nbx=32, nby=32, wdtype=2, ntaps=3, tap_k=(2, 4, 8, 0),
                       tap_alpha=(1 / 3, 1 / 3, 1 / 3, 0)), (0, 2, 4), 2),
    # the 2.2M-cell workload with a committed model's parameters and powers
    pytest.param("large", 1, dict(nbx=32, nby=32, wdtype=2, ntaps=3, tap_k=(2, 4, 8, 0),
                                  tap_alpha=(1 / 3, 1 / 3, 1 / 3, 0), pin_every_step=1),
                 (0, 1, 2), 1, marks=pytest.mark.slow)])
def test_learned_round_matches_oracle(cfg, seed, kw, k, rnd):
    m = pl()
    s = Round(cfg, seed, **kw)
    w, _ = random_model(9, w1=0.3, w2=0.02, theta=(0.2, -0.5, 1.3))
    model = m.LearnedModel(k, dev(w))
    out = torch.full_like(s.xy, float("nan"))
    m.pl_learned_apply(s.g, s.prm, model, rnd, s.xy, out)
    torch.cuda.synchronize()
    got = out.view(-1, 2).double().cpu().numpy()
    want, _ = L.learned_round(s.o, s.ax, s.ay, k, rnd, w.astype(np.float64))
    err = np.abs(got - want).max()
    assert err <= 1e-4 * s.die, err
    # the round moved the free nodes (the check is not vacuous)
    assert np.abs(want - np.stack([s.ax, s.ay], 1)).max() > 1e-3 * s.die


# ------------------------------------------------------------- training
def seeded_records(seed, n, taps=None):
    """Records [n, 24] (FP32 values): features, taps and targets of the
    shapes a round produces (taps near each other, targets near the taps)."""
    rng = np.random.default_rng(seed)
    f = rng.normal(0, 1, (n, L.NF)) * rng.uniform(0.1, 3.0, L.NF)
    f[:, 8] = rng.random(n) < 0.9
    f[:, 9] = 1 - f[:, 8]
    f[:, 11] = 0.5
    f[:, 12:] = 0
    G0 = rng.normal(0, 5, (n, 2))
    G1 = G0 + rng.normal(0, 1.0, (n, 2))
    G2 = 0.5 * G0 + rng.normal(0, 1.0, (n, 2))
    th = (0.3, -0.4, 1.1) if taps is None else taps
    T = th[0] * G0 + th[1] * G1 + th[2] * G2 + rng.normal(0, 0.3, (n, 2))
    R = np.concatenate([f, G0, G1, G2, T], 1).astype(np.float32)
    return R


def split(R):
    R = R.astype(np.float64)
    return R[:, 16:18], R[:, 18:20], R[:, 20:22], R[:, 0:16], R[:, 22:24]


def test_loss_and_gradient_match_oracle():
    m = pl()
    R = seeded_records(21, 128 * 9 + 50)
    w, p = random_model(7, w1=0.3, w2=0.2)
    grad = torch.full((m.LEARNED_SIZE,), float("nan"), device="cuda")
    loss = m.pl_learned_loss(dev(R.reshape(-1)), len(R), dev(w), grad)
    G0, G1, G2, f, T = split(R)
    want, gr = L.loss_and_grads(p, G0, G1, G2, f, T)
    assert loss == pytest.approx(want, rel=1e-4)
    g = grad.double().cpu().numpy()
    assert np.all(g[:L.THETA] == 0)
    got = L.unpack(g)
    for k in L.TRAINED:
        a, b = np.asarray(got[k]), np.asarray(gr[k])
        assert np.abs(a - b).max() <= 1e-3 * np.abs(b).max() + 1e-7, (k, np.abs(a - b).max(), np.abs(b).max())


def test_one_adam_step_matches_oracle():
    m = pl()
    R = seeded_records(22, 1024)
    w, p = random_model(8, w1=0.3, w2=0.2)
    model = m.LearnedModel((0, 1, 2), dev(w))
    lr = 1e-3
    o = m.train_opts(epochs=1, batch_tiles=8, lr=lr, lr_min=lr, fit_norm=0, fit_taps=0, seed=3)
    hist = m.pl_learned_train(dev(R.reshape(-1)), len(R), model, o)
    wn = model.w.double().cpu().numpy()
    G0, G1, G2, f, T = split(R)
    loss, gr = L.loss_and_grads(p, G0, G1, G2, f, T)
    assert hist[0] == pytest.approx(loss, rel=1e-4)
    q = {k: np.array(v, copy=True) for k, v in p.items()}
    mm = {k: np.zeros_like(v) for k, v in q.items()}
    vv = {k: np.zeros_like(v) for k, v in q.items()}
    L.adam_step(q, gr, mm, vv, 1, lr=lr)
    got, w0 = L.unpack(wn), L.unpack(w.astype(np.float64))
    assert np.array_equal(wn[:L.THETA], w[:L.THETA].astype(np.float64))  # normalisation kept
    for k in L.TRAINED:
        step_gpu = np.asarray(got[k]) - np.asarray(w0[k])
        step_orc = np.asarray(q[k]) - np.asarray(w0[k])
        big = np.abs(gr[k]) > 1e-3 * np.abs(gr[k]).max()
        assert np.abs(step_gpu - step_orc)[big].max() <= 2e-3 * lr, k
        assert np.abs(step_gpu).max() <= lr * (1 + 1e-3), k  # a first Adam step is at most lr


def test_fitted_normalisation_and_taps_match_oracle():
    m = pl()
    R = seeded_records(23, 128 * 6, taps=(0.3, -0.4, 1.1))
    w, _ = random_model(9)
    model = m.LearnedModel((0, 1, 2), dev(w))
    o = m.train_opts(epochs=1, batch_tiles=6, lr=1e-30, lr_min=1e-30)
    m.pl_learned_train(dev(R.reshape(-1)), len(R), model, o)
    got = L.unpack(model.w.double().cpu().numpy())
    G0, G1, G2, f, T = split(R)
    mu, isd = L.fit_norm(f)
    th = L.fit_taps(G0, G1, G2, T)
    assert np.abs(got["mu"] - mu).max() <= 1e-6 * (1 + np.abs(mu)).max()
    assert np.allclose(got["isd"], isd, rtol=1e-5)
    assert np.all(got["isd"][11:] == 1.0)
    assert np.allclose(got["theta"], th, rtol=1e-5)


def test_training_reduces_the_loss_and_is_reproducible():
    m = pl()
    R = dev(seeded_records(24, 128 * 40).reshape(-1))
    runs = []
    for _ in range(2):
        model = m.learned_init((0, 1, 2), 5)
        hist = m.pl_learned_train(R, 128 * 40, model, m.train_opts(epochs=6, batch_tiles=8, seed=4))
        runs.append((hist, model.w.cpu().numpy()))
    assert runs[0][0][-1] < runs[0][0][0]
    assert runs[0][0] == runs[1][0] and np.array_equal(runs[0][1], runs[1][1])


# ------------------------------------------------- the whole initializer
def test_initializer_without_model_and_fallback_are_the_plain_bits():
    m = pl()
    nl = netgen.make_netlist("tiny", 4)
    prm = m.params(nbx=16, nby=16)
    g = m.pl_build_graph(m.DeviceNetlist(nl), prm)
    C = nl.num_cells
    plain = torch.empty(C * 2, device="cuda")
    m.pl_filter_init(g, prm, 4, None, plain)
    out = torch.full_like(plain, float("nan"))
    assert m.pl_filter_init_learned(g, prm, None, 4, None, out) == 0
    assert torch.equal(out, plain)
    # a model whose output is NaN: every round falls back to the plain filter
    w, _ = random_model(3)
    w[L.B2] = np.nan
    bad = m.LearnedModel((0, 1, 2), dev(w))
    out.fill_(float("nan"))
    assert m.pl_filter_init_learned(g, prm, bad, 4, None, out) == prm.t_hint
    assert torch.equal(out, plain)
    with pytest.raises(m.PlError) as e:
        m.pl_learned_apply(g, prm, bad, 0, torch.zeros(g.info()["N"] * 2, device="cuda"),
                           torch.empty(g.info()["N"] * 2, device="cuda"))
    assert e.value.code == m.PL_ERR_NONFINITE
    # a finite model: no fallback, a placement inside the region
    w, _ = random_model(3, w2=0.02, theta=(0.2, -0.5, 1.3))
    good = m.LearnedModel((0, 2, 4), dev(w))
    assert m.pl_filter_init_learned(g, prm, good, 4, None, out) == 0
    xy = out.view(-1, 2).cpu().numpy()
    mov = np.asarray(nl.cell_kind) == 0
    xl, yl, xh, yh = nl.region
    assert np.isfinite(xy).all()
    assert (xy[mov, 0] >= xl).all() and (xy[mov, 0] <= xh).all()
    assert (xy[mov, 1] >= yl).all() and (xy[mov, 1] <= yh).all()
    assert not torch.equal(out, plain)


def test_learned_argument_errors():
    m = pl()
    nl = netgen.make_netlist("micro", 1)
    prm = m.params(nbx=4, nby=4)
    g = m.pl_build_graph(m.DeviceNetlist(nl), prm)
    N = g.info()["N"]
    w, _ = random_model(1)
    x = torch.zeros(N * 2, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(m.PlError) as e:  # no hints built yet
        m.pl_learned_apply(g, prm, m.LearnedModel((0, 1, 2), dev(w)), 0, x, y)
    assert e.value.code == m.PL_ERR_INVALID_ARG
    for k in ((1, 1, 2), (0, 3, 2), (-1, 1, 2), (0, 1, 65)):
        with pytest.raises(m.PlError) as e:
            m.pl_filter_init_learned(g, prm, m.LearnedModel(k, dev(w)), 1, None, y)
        assert e.value.code == m.PL_ERR_INVALID_ARG, k
    R = dev(seeded_records(1, 100).reshape(-1))
    with pytest.raises(m.PlError) as e:  # fewer than one tile of records
        m.pl_learned_train(R, 100, m.LearnedModel((0, 1, 2), dev(w)), m.train_opts())
    assert e.value.code == m.PL_ERR_INVALID_ARG


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    """The tensor-core kernels' mbarrier waits are bounded: a wait on a phase
    that nothing completes gives up after the limit (about 1 ms here), the
    CTA frees its tensor memory, and the host reads PL_ERR_TIMEOUT.  The
    tensor-core path then still gives exact results."""
    m = pl()
    import time
    t0 = time.perf_counter()
    assert m.pl_learned_wait_check(2_000_000) == m.PL_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 30
    assert "gave up" in m.lib().pl_last_error().decode()
    test_forward_exact_on_dyadic_inputs()
