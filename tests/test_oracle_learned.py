"""Pins of the learned-filter oracle (oracle/learned.py): BF16 rounding
against torch's, the gradients against finite differences of the unrounded
forward, features and prediction in closed cases, one Adam step by hand."""
import numpy as np
import pytest

from oracle import learned as L

torch = pytest.importorskip("torch")


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(1)
    a = np.r_[rng.normal(0, 3, 5000), rng.normal(0, 1e-30, 100), [0.0, -0.0, 1.0, 65504.0, 3.0e38]]
    want = torch.tensor(a, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(L.bf16(a), want)


def _setup(seed=3, N=40):
    rng = np.random.default_rng(seed)
    p = {"theta": rng.normal(0, 0.5, 3), "W1": rng.normal(0, 0.3, (L.HID, L.NF)),
         "b1": rng.normal(0, 0.1, L.HID), "W2": rng.normal(0, 0.3, (2, L.HID)),
         "b2": rng.normal(0, 0.1, 2)}
    g = rng.normal(50, 10, (N, 2))
    hg = g + rng.normal(0, 1, (N, 2))
    h2g = g + rng.normal(0, 2, (N, 2))
    f = rng.normal(0, 1, (N, L.NF))
    target = g + rng.normal(0, 3, (N, 2))
    mov = rng.random(N) < 0.8
    return p, g, hg, h2g, f, target, mov


def test_gradients_against_finite_differences(monkeypatch):
    # the unrounded forward (bf16 as identity): the gradient formulas are the
    # exact derivative there
    monkeypatch.setattr(L, "bf16", lambda a: np.asarray(a, np.float64))
    p, g, hg, h2g, f, target, mov = _setup()
    sx, sy = 2.5, 4.0
    loss, gr = L.loss_and_grads(p, g, hg, h2g, f, target, mov, sx, sy)
    rng = np.random.default_rng(0)
    for k in p:
        for _ in range(6):
            idx = tuple(rng.integers(0, d) for d in p[k].shape)
            h = 1e-6
            q = {kk: vv.copy() for kk, vv in p.items()}
            q[k][idx] += h
            lp, _ = L.loss_and_grads(q, g, hg, h2g, f, target, mov, sx, sy)
            q[k][idx] -= 2 * h
            lm, _ = L.loss_and_grads(q, g, hg, h2g, f, target, mov, sx, sy)
            fd = (lp - lm) / (2 * h)
            assert gr[k][idx] == pytest.approx(fd, rel=1e-5, abs=1e-8), (k, idx)


def test_features_on_a_constant_signal():
    N = 6
    g = np.full((N, 2), 7.0)
    deg = np.array([2.0, 1.0, -0.5, 3.0, 0.0, 1.5])
    psum = np.array([2.0, 1.0, 0.5, 3.5, 0.0, 1.5])
    hint = np.array([True, False, True, True, False, False])
    phi = np.array([0.3, 0.9, -0.2, 0.1, 0.0, 0.0])
    f = L.features(g, g, g, deg, psum, 4.0, hint, phi, 2.0, 3.0)
    assert np.all(f[:, 0:4] == 0.0)  # H preserves constants
    assert np.allclose(f[:, 4], 1 - deg / 4.0)
    assert np.allclose(f[:, 5], (2 * psum - deg) / 4.0)  # sum of |w|
    assert np.allclose(f[:, 6], (deg - psum) / 4.0)      # sum of negative w
    assert np.array_equal(f[:, 7], np.where(hint, phi, 0.0))
    assert np.array_equal(f[:, 8], hint.astype(float)) and np.all(f[:, 9:] == 0)


def test_prediction_reduces_to_a_tap():
    p, g, hg, h2g, f, target, mov = _setup()
    _, _, out = L.mlp_forward(f, p["W1"], p["b1"], np.zeros((2, L.HID)), np.zeros(2))
    assert np.all(out == 0.0)
    assert np.array_equal(L.predict(np.array([0.0, 0.0, 1.0]), g, hg, h2g, out, 2.0, 3.0), h2g)
    assert np.array_equal(L.predict(np.array([1.0, 0.0, 0.0]), g, hg, h2g, out, 2.0, 3.0), g)


def test_one_adam_step_by_hand():
    p = {"a": np.array([1.0, -2.0, 0.5])}
    gr = {"a": np.array([0.1, -4.0, 0.0])}
    m, v = {"a": np.zeros(3)}, {"a": np.zeros(3)}
    L.adam_step(p, gr, m, v, 1, lr=0.01)
    # first step: m^ = g, v^ = g^2, update lr g / (|g| + eps)
    want = np.array([1.0, -2.0, 0.5]) - 0.01 * gr["a"] / (np.abs(gr["a"]) + 1e-8)
    assert np.allclose(p["a"], want, rtol=1e-12)
