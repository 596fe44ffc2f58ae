"""FP64 statement of the learned refinement filter (TEST INFRASTRUCTURE ONLY).

The refinement filter of Sec. V applies H_r^k, H_r = I - L_hint / lambda_up,
with k = 8 in the plain initializer.  The learned filter stands in for it with
two products and a per-node correction:

    g~ = theta_0 g + theta_1 H g + theta_2 H^2 g + s * MLP(f),

s the bin size per axis, f a node's 16 features and MLP a two-layer
perceptron 16 -> 64 (ReLU) -> 2.  It is trained to match the plain order-8
filter H^8 g on the movable cells (the plain filter stays the judge).  This
module states every step in plain numpy, FP64, with the BF16 roundings the
GPU's tensor cores see (features, weights, hidden layer) written out, so that
the CUDA kernels can be compared with it.  Only the tests and the benchmark's
evaluation may import it.
"""
from __future__ import annotations

import numpy as np

NF = 16   # features per node
HID = 64  # hidden units


def bf16(a):
    """Round to bfloat16 (8 significant bits), nearest even, kept as float64."""
    a = np.asarray(a, np.float64).astype(np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(a)
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def features(g, hg, h2g, deg, psum, lam, hint, phi_own, sx, sy):
    """The 16 features of every node (rows), as the learned filter defines them:
      0, 1  (H g - g) per axis over the bin size
      2, 3  (H^2 g - g) per axis over the bin size
      4     the diagonal of H, 1 - D_vv / lambda_up
      5     the row's absolute weight, sum_j |w_vj| = 2 P_v - D_vv, over lambda_up
      6     the row's negative weight, D_vv - P_v, over lambda_up
      7     phi of the node's bin (hint cells), else 0
      8     1 for a hint cell, else 0
      9-15  0
    g, hg, h2g: [N, 2]; deg, psum: [N] signed degree and positive-weight sum."""
    N = g.shape[0]
    f = np.zeros((N, NF))
    s = np.array([sx, sy])
    f[:, 0:2] = (hg - g) / s
    f[:, 2:4] = (h2g - g) / s
    f[:, 4] = 1.0 - deg / lam
    f[:, 5] = (2.0 * psum - deg) / lam
    f[:, 6] = (deg - psum) / lam
    f[:, 7] = np.where(hint, phi_own, 0.0)
    f[:, 8] = np.where(hint, 1.0, 0.0)
    return f


def mlp_forward(f, W1, b1, W2, b2):
    """Two layers as the tensor cores compute them: BF16 features times BF16
    W1 (64 x 16) plus b1, ReLU, the hidden layer rounded to BF16, times BF16
    W2 (2 x 64) plus b2.  Returns (pre-activation, hidden, output [N, 2])."""
    x = bf16(f)
    pre = x @ bf16(W1).T + b1
    h = np.maximum(pre, 0.0)
    hb = bf16(h)
    out = hb @ bf16(W2).T + b2
    return pre, hb, out


def predict(theta, g, hg, h2g, out, sx, sy):
    """theta_0 g + theta_1 H g + theta_2 H^2 g + s * MLP output."""
    s = np.array([sx, sy])
    return theta[0] * g + theta[1] * hg + theta[2] * h2g + s * out


def loss_and_grads(params, g, hg, h2g, f, target, mov, sx, sy):
    """Mean over movable cells of the squared error in bin units,
    sum over axes of ((pred - target) / s)^2, and its gradients with respect
    to theta, W1, b1, W2, b2 (the BF16 roundings treated as identity, the
    straight-through reading)."""
    theta, W1, b1, W2, b2 = (params[k] for k in ("theta", "W1", "b1", "W2", "b2"))
    pre, hb, out = mlp_forward(f, W1, b1, W2, b2)
    s = np.array([sx, sy])
    pred = predict(theta, g, hg, h2g, out, sx, sy)
    e = np.where(mov[:, None], (pred - target) / s, 0.0)
    n = max(int(mov.sum()), 1)
    loss = float((e * e).sum() / n)
    de = 2.0 * e / n                      # d loss / d ((pred - target) / s)
    dpred = de / s
    gt = np.array([(dpred * g).sum(), (dpred * hg).sum(), (dpred * h2g).sum()])
    dout = dpred * s                      # pred = ... + s * out
    dW2 = dout.T @ hb
    db2 = dout.sum(0)
    dh = (dout @ bf16(W2)) * (pre > 0.0)
    dW1 = dh.T @ bf16(f)
    db1 = dh.sum(0)
    return loss, {"theta": gt, "W1": dW1, "b1": db1, "W2": dW2, "b2": db2}


def adam_step(params, grads, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba) on every parameter array, t >= 1."""
    for k in params:
        m[k] = beta1 * m[k] + (1 - beta1) * grads[k]
        v[k] = beta2 * v[k] + (1 - beta2) * grads[k] * grads[k]
        mh = m[k] / (1 - beta1 ** t)
        vh = v[k] / (1 - beta2 ** t)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)
    return params
