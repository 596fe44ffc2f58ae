"""Pins of the learned-filter oracle (oracle/learned.py): BF16 rounding
against torch's, the gradients against finite differences of the unrounded
forward, features, normalisation, least-squares taps and the round's end in
closed cases, one Adam step by hand, and the learned round with a pure-tap
model against the plain filter of the C oracle."""
import numpy as np
import pytest

import oracle
from oracle import learned as L
from paper_2511_10073_gb300 import netgen

torch = pytest.importorskip("torch")


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(1)
    a = np.r_[rng.normal(0, 3, 5000), rng.normal(0, 1e-30, 100), [0.0, -0.0, 1.0, 65504.0, 3.0e38]]
    want = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(L.bf16(a), want)


def _params(rng):
    return {"mu": rng.normal(0, 0.2, L.NF), "isd": rng.uniform(0.5, 2.0, L.NF),
            "theta": rng.normal(0, 0.5, 3), "W1": rng.normal(0, 0.3, (L.HID, L.NF)),
            "b1": rng.normal(0, 0.1, L.HID), "W2": rng.normal(0, 0.3, (L.NOUT, L.HID)),
            "b2": rng.normal(0, 0.1, L.NOUT)}


def _records(rng, n=40):
    G0 = rng.normal(3, 4, (n, 2))
    G1 = G0 + rng.normal(0, 0.3, (n, 2))
    G2 = G0 + rng.normal(0, 0.5, (n, 2))
    f = rng.normal(0, 1, (n, L.NF))
    T = G0 + rng.normal(0, 0.6, (n, 2))
    return G0, G1, G2, f, T


def test_pack_unpack_round_trip():
    p = _params(np.random.default_rng(2))
    q = L.unpack(L.pack(p))
    for k in p:
        assert np.array_equal(np.asarray(p[k]), q[k]), k
    assert L.SIZE == 16 + 16 + 3 + L.HID * L.NF + L.HID + L.NOUT * L.HID + L.NOUT


def test_gradients_against_finite_differences(monkeypatch):
    # the unrounded forward (bf16 as identity): the gradient formulas are the
    # exact derivative there
    monkeypatch.setattr(L, "bf16", lambda a: np.asarray(a, np.float64))
    rng = np.random.default_rng(3)
    p = _params(rng)
    G0, G1, G2, f, T = _records(rng)
    mask = rng.random(len(G0)) < 0.8
    loss, gr = L.loss_and_grads(p, G0, G1, G2, f, T, mask)
    for k in L.TRAINED:
        for _ in range(6):
            idx = tuple(rng.integers(0, d) for d in np.shape(p[k]))
            h = 1e-6
            q = {kk: np.array(vv, copy=True) for kk, vv in p.items()}
            q[k][idx] += h
            lp, _ = L.loss_and_grads(q, G0, G1, G2, f, T, mask)
            q[k][idx] -= 2 * h
            lm, _ = L.loss_and_grads(q, G0, G1, G2, f, T, mask)
            fd = (lp - lm) / (2 * h)
            assert gr[k][idx] == pytest.approx(fd, rel=1e-5, abs=1e-8), (k, idx)


def test_features_in_closed_cases():
    N = 6
    G = np.full((N, 2), 7.0)
    deg = np.array([2.0, 1.0, -0.5, 3.0, 0.0, 1.5])
    psum = np.array([2.0, 1.0, 0.5, 3.5, 0.0, 1.5])
    hint = np.array([True, False, True, True, False, False])
    star = np.array([False, False, False, False, True, False])
    phi = np.array([0.3, 0.9, -0.2, 0.1, 0.0, 0.0])
    area = np.array([0.5, 0.25, 0.0, 1.0, 0.0, 0.0])
    f = L.features(G, G, G, deg, psum, 4.0, hint, phi, star, area, 2 / 3)
    assert np.all(f[:, 0:4] == 0.0)  # a constant signal has no tap steps
    assert np.allclose(f[:, 4], deg / 4.0)
    assert np.allclose(f[:, 5], (2 * psum - deg) / 4.0)  # sum of |w|: P + (P - D)
    assert np.allclose(f[:, 6], (deg - psum) / 4.0)      # sum of the negative w
    assert np.array_equal(f[:, 7], np.where(hint, phi, 0.0))
    assert np.array_equal(f[:, 8], hint.astype(float))
    assert np.array_equal(f[:, 9], star.astype(float))
    assert np.array_equal(f[:, 10], area) and np.all(f[:, 11] == 2 / 3) and np.all(f[:, 12:] == 0)
    G1 = G + np.array([1.5, -2.0])
    G2 = G + np.array([-0.25, 4.0])
    f = L.features(G, G1, G2, deg, psum, 4.0, hint, phi, star, area, 0.0)
    assert np.all(f[:, 0:2] == [1.5, -2.0]) and np.all(f[:, 2:4] == [-0.25, 4.0])


def test_normalisation_standardises():
    rng = np.random.default_rng(4)
    f = rng.normal(5, 3, (5000, L.NF))
    f[:, 12:] = 0.0
    f[:, 11] = 0.5
    mu, isd = L.fit_norm(f)
    z = (f - mu) * isd
    assert np.allclose(z[:, :11].mean(0), 0, atol=1e-12)
    assert np.allclose(z[:, :11].std(0), 1, rtol=1e-12)
    assert np.all(isd[11:] == 1.0) and np.all(z[:, 11:] == 0.0)
    x = L.normalise(f, mu, isd)
    assert np.array_equal(x, L.bf16(z))


def test_fit_taps_recovers_an_exact_combination():
    rng = np.random.default_rng(5)
    G0, G1, G2, f, T = _records(rng, 200)
    th = np.array([0.3, -1.2, 1.9])
    assert np.allclose(L.fit_taps(G0, G1, G2, th[0] * G0 + th[1] * G1 + th[2] * G2), th, rtol=1e-10)


def test_prediction_in_closed_cases():
    rng = np.random.default_rng(6)
    G0, G1, G2, f, T = _records(rng)
    zero = np.zeros((len(G0), L.NOUT))
    assert np.array_equal(L.predict(np.array([0.0, 0.0, 1.0]), G0, G1, G2, zero), G2)
    assert np.array_equal(L.predict(np.array([1.0, 0.0, 0.0]), G0, G1, G2, zero), G0)
    # a = 1 turns tap G0 into G1; b = 1 turns it into G2; o shifts
    one = zero.copy(); one[:, 0] = 1.0
    assert np.allclose(L.predict(np.array([1.0, 0.0, 0.0]), G0, G1, G2, one), G1)
    one = zero.copy(); one[:, 1] = 1.0; one[:, 2:4] = [0.5, -0.25]
    assert np.allclose(L.predict(np.array([1.0, 0.0, 0.0]), G0, G1, G2, one), G2 + [0.5, -0.25])
    # the MLP with W2 = 0 outputs b2 on every node
    p = _params(rng)
    p["W2"][:] = 0.0
    _, _, out = L.mlp_forward(L.normalise(f, p["mu"], p["isd"]), p)
    assert np.all(out == p["b2"])


def test_one_adam_step_by_hand():
    p = {k: np.array([1.0, -2.0, 0.5]) if k == "theta" else np.zeros(1) for k in L.TRAINED}
    gr = {k: np.array([0.1, -4.0, 0.0]) if k == "theta" else np.zeros(1) for k in L.TRAINED}
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(x) for k, x in p.items()}
    L.adam_step(p, gr, m, v, 1, lr=0.01)
    # first step: m^ = g, v^ = g^2, update lr g / (|g| + eps)
    want = np.array([1.0, -2.0, 0.5]) - 0.01 * gr["theta"] / (np.abs(gr["theta"]) + 1e-8)
    assert np.allclose(p["theta"], want, rtol=1e-12)


def test_finish_round():
    nk = np.array([0, 1, 2, 0], np.uint8)
    fx, fy = np.array([0, 0, 5.0, 0]), np.array([0, 0, 6.0, 0])
    hw, hh = np.array([1.0, 0.0, 3.0, 0.5]), np.array([2.0, 0.0, 3.0, 0.5])
    g = np.array([[2.0, 3.0], [4.0, 4.0], [9.0, 9.0], [9.5, 1.0]])
    gt = np.array([[4.0, 5.0], [-2.0, 6.0], [0.0, 0.0], [9.9, 9.9]])
    o = L.finish_round(gt, g, nk, fx, fy, hw, hh, (0.0, 0.0, 10.0, 10.0), 0.5, 1)
    assert np.array_equal(o, [[3.0, 4.0], [1.0, 5.0], [5.0, 6.0], [9.5, 5.45]])


def test_pure_tap_model_is_the_plain_filter():
    """theta = (0, 0, 1) and a zero MLP at powers (0, 1, 2) is the plain
    filter H_r^2: the learned round's taps, bin-unit transforms and round end
    reproduce the C oracle's filter-and-relax step."""
    nl = netgen.make_netlist("tiny", 3)
    prm = dict(nbx=16, nby=16, ntaps=1, tap_k=(2, 0, 0, 0), tap_alpha=(1.0, 0, 0, 0))
    o = oracle.Oracle(nl, **prm)
    gx, gy = o.init_signal(3)
    gx, gy = o.gift(gx, gy)
    o.build_hints(gx, gy)
    w = np.zeros(L.SIZE)
    w[L.ISD:L.ISD + L.NF] = 1.0
    w[L.THETA + 2] = 1.0
    g1, gt = L.learned_round(o, gx, gy, (0, 1, 2), 0, w)
    ox, oy = o.filter(gx, gy)
    die = nl.region[2] - nl.region[0]
    assert np.max(np.abs(g1 - np.stack([ox, oy], 1))) < 1e-9 * die
    # the learned round's taps are the C oracle's powers
    r = L.round_inputs(o, gx, gy, (0, 1, 2), 0)
    h2 = o.hr_steps(2, gx)
    assert np.allclose(r["c"][0] + r["s"][0] * r["G2"][:, 0], h2, rtol=0, atol=1e-9 * die)


def test_effective_target_inverts_the_relaxation():
    rng = np.random.default_rng(8)
    nk = np.array([0, 1, 0, 0], np.uint8)
    g = rng.uniform(2, 8, (4, 2))
    gt = rng.uniform(2, 8, (4, 2))
    z = np.zeros(4)
    for gamma in (0.3, 0.5, 1.0):
        g1 = L.finish_round(gt, g, nk, z, z, z, z, (0.0, 0.0, 10.0, 10.0), gamma, 1)
        assert np.allclose(L.effective_target(g1, g, gamma), gt, rtol=1e-13)
    # where the clamp acted the target is the output that relaxes onto the edge
    gt[0] = [40.0, -30.0]
    g1 = L.finish_round(gt, g, nk, z, z, z, z, (0.0, 0.0, 10.0, 10.0), 0.5, 1)
    t = L.effective_target(g1, g, 0.5)
    assert np.allclose(0.5 * g[0] + 0.5 * t[0], [10.0, 0.0])
