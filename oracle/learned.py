"""FP64 statement of the learned refinement filter (TEST INFRASTRUCTURE ONLY).

The refinement filter of Sec. V (Algorithm 1, step "filter") applies a
polynomial in H_r = I - L_hint / lambda_up of high order (taps up to H_r^8 in
the plain initializer), one sparse product per power.  The learned filter
stands in for it with three taps at lower powers k0 < k1 < k2 and a per-node
correction.  In bin units about the region centre c (s the bin size per
axis), with G_t = (H_r^{k_t} g - c) / s:

    P_v = theta_0 G0 + theta_1 G1 + theta_2 G2
          + a_v (G1 - G0) + b_v (G2 - G0) + (o_v^x, o_v^y),
    (a_v, b_v, o_v^x, o_v^y) = MLP(x_v),   g~_v = c + s P_v,

the MLP two layers 16 -> 64 (ReLU) -> 4 on the node's normalised features
x_v.  The rest of the round is the plain filter's (fixed nodes re-pinned,
relaxation by gamma, re-pinned, movable centres clamped).  It is trained to
reproduce the plain round (the plain filter stays the judge): its target is
the filter output that the relaxation maps to the plain round's result g',
(g' - (1 - gamma) g) / gamma, which is the plain g~ wherever clamping did not
act (the signed graph's H_r can amplify, so an unclamped g~ may lie far
outside the region; the clamped result is what the round keeps).

Every step is written in plain numpy, FP64, with the BF16 roundings that the
GPU's tensor cores see (normalised features, weights, hidden layer) written
out.  Only the tests and the benchmark's evaluation may import this module.
"""
from __future__ import annotations

import numpy as np

NF = 16    # features per node
HID = 64   # hidden units
NOUT = 4   # MLP outputs: a, b, o^x, o^y

# Layout of the parameter vector (FP32 on the device; float64 here).
MU, ISD, THETA = 0, 16, 32
W1 = 35                    # [HID][NF]
B1 = W1 + HID * NF         # [HID]
W2 = B1 + HID              # [NOUT][HID]
B2 = W2 + NOUT * HID       # [NOUT]
SIZE = B2 + NOUT


def bf16(a):
    """Round to bfloat16 (8 significant bits), nearest even, through FP32
    (FP64 -> FP32 -> BF16, each rounding to nearest even); kept as float64."""
    a = np.asarray(a, np.float64).astype(np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    nan = np.isnan(a)
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    out[nan] = np.nan
    return out


def unpack(w):
    """The parameter vector as named arrays (views)."""
    w = np.asarray(w, np.float64)
    return dict(mu=w[MU:MU + NF], isd=w[ISD:ISD + NF], theta=w[THETA:THETA + 3],
                W1=w[W1:B1].reshape(HID, NF), b1=w[B1:W2], W2=w[W2:B2].reshape(NOUT, HID),
                b2=w[B2:SIZE])


def pack(p):
    w = np.zeros(SIZE)
    w[MU:MU + NF] = p["mu"]
    w[ISD:ISD + NF] = p["isd"]
    w[THETA:THETA + 3] = p["theta"]
    w[W1:B1] = np.asarray(p["W1"]).ravel()
    w[B1:W2] = p["b1"]
    w[W2:B2] = np.asarray(p["W2"]).ravel()
    w[B2:SIZE] = p["b2"]
    return w


def effective_target(g1, g, gamma):
    """The filter output that the relaxation maps to the round result g1:
    (g1 - (1 - gamma) g) / gamma, gamma > 0."""
    return (np.asarray(g1, np.float64) - (1.0 - gamma) * np.asarray(g, np.float64)) / gamma


def bins(xy, c, s):
    """Coordinates [N, 2] in bin units about the centre c."""
    return (np.asarray(xy, np.float64) - c) / s


def features(G0, G1, G2, deg, psum, lam, hint, phi_own, star, area, rnd):
    """The 16 raw features of every node (rows):
      0, 1  G1 - G0 per axis (the first tap step, bin units)
      2, 3  G2 - G0 per axis
      4     D_vv / lambda_up (signed degree)
      5     sum_j |w_vj| / lambda_up = (2 P_v - D_vv) / lambda_up, P_v the
            row's positive-weight sum
      6     (D_vv - P_v) / lambda_up, the row's negative weights
      7     phi_b of a hint cell's own bin (Sec. V bin hints), else 0
      8     1 for a hint cell (movable, baseWeight > 0), else 0
      9     1 for a star node, else 0
      10    a movable cell's area over the bin area, else 0
      11    the round t / T_hint of Algorithm 1
      12-15 0"""
    N = G0.shape[0]
    f = np.zeros((N, NF))
    f[:, 0:2] = G1 - G0
    f[:, 2:4] = G2 - G0
    f[:, 4] = deg / lam
    f[:, 5] = (2.0 * psum - deg) / lam
    f[:, 6] = (deg - psum) / lam
    f[:, 7] = np.where(hint, phi_own, 0.0)
    f[:, 8] = np.where(hint, 1.0, 0.0)
    f[:, 9] = np.where(star, 1.0, 0.0)
    f[:, 10] = area
    f[:, 11] = rnd
    return f


def normalise(f, mu, isd):
    """The MLP input: (f - mu) * isd per feature, rounded to BF16."""
    return bf16((f - mu) * isd)


def fit_norm(f):
    """Feature mean and inverse standard deviation over the records (1 where
    a feature is constant)."""
    mu = f.mean(0)
    sd = np.sqrt(np.maximum((f * f).mean(0) - mu * mu, 0.0))
    isd = np.where(sd > 1e-12 * (1.0 + np.abs(mu)), 1.0 / np.where(sd > 0, sd, 1.0), 1.0)
    return mu, isd


def fit_taps(G0, G1, G2, T):
    """Least-squares taps: theta minimising sum ||theta . (G0, G1, G2) - T||^2
    over records and both axes (the normal equations)."""
    A = np.stack([G0.ravel(), G1.ravel(), G2.ravel()], 1)
    return np.linalg.solve(A.T @ A, A.T @ T.ravel())


def mlp_forward(x, p):
    """Two layers as the tensor cores compute them: BF16 inputs x times BF16
    W1 (64 x 16) plus b1, ReLU, the hidden layer rounded to BF16, times BF16
    W2 (4 x 64) plus b2.  Returns (pre-activation, hidden, output [N, 4])."""
    pre = x @ bf16(p["W1"]).T + p["b1"]
    hb = bf16(np.maximum(pre, 0.0))
    out = hb @ bf16(p["W2"]).T + p["b2"]
    return pre, hb, out


def predict(theta, G0, G1, G2, out):
    """P = theta . (G0, G1, G2) + a (G1 - G0) + b (G2 - G0) + o, bin units."""
    return (theta[0] * G0 + theta[1] * G1 + theta[2] * G2 + out[:, 0:1] * (G1 - G0)
            + out[:, 1:2] * (G2 - G0) + out[:, 2:4])


def loss_and_grads(p, G0, G1, G2, f, T, mask=None):
    """Mean over the masked records of the squared error summed over both
    axes, sum ((P - T))^2 in bin units, and its gradients with respect to
    theta, W1, b1, W2, b2 (the BF16 roundings treated as identity: the
    straight-through reading).  f: raw features."""
    n_all = G0.shape[0]
    m = np.ones(n_all, bool) if mask is None else np.asarray(mask, bool)
    x = normalise(f, p["mu"], p["isd"])
    pre, hb, out = mlp_forward(x, p)
    P = predict(p["theta"], G0, G1, G2, out)
    e = np.where(m[:, None], P - T, 0.0)
    n = max(int(m.sum()), 1)
    loss = float((e * e).sum() / n)
    dP = 2.0 * e / n
    gt = np.array([(dP * G0).sum(), (dP * G1).sum(), (dP * G2).sum()])
    dout = np.zeros((n_all, NOUT))
    dout[:, 0] = (dP * (G1 - G0)).sum(1)
    dout[:, 1] = (dP * (G2 - G0)).sum(1)
    dout[:, 2:4] = dP
    dW2 = dout.T @ hb
    db2 = dout.sum(0)
    dh = (dout @ bf16(p["W2"])) * (pre > 0.0)
    dW1 = dh.T @ x
    db1 = dh.sum(0)
    return loss, {"theta": gt, "W1": dW1, "b1": db1, "W2": dW2, "b2": db2}


TRAINED = ("theta", "W1", "b1", "W2", "b2")


def adam_step(p, grads, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba, Algorithm 1) on every trained array, t >= 1."""
    for k in TRAINED:
        m[k] = beta1 * m[k] + (1 - beta1) * grads[k]
        v[k] = beta2 * v[k] + (1 - beta2) * grads[k] * grads[k]
        mh = m[k] / (1 - beta1 ** t)
        vh = v[k] / (1 - beta2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return p


def finish_round(gt, g, nkind, fx, fy, hw, hh, region, gamma, clamp):
    """The end of a refinement round on the filter output gt [N, 2] (the
    plain filter's, and the learned filter's): fixed nodes re-pinned,
    g' = (1 - gamma) g + gamma g~, re-pinned, movable centres (and star
    nodes, as points) clamped into the region."""
    fixed = nkind == 2
    gt = np.array(gt, np.float64)
    gt[fixed, 0], gt[fixed, 1] = fx[fixed], fy[fixed]
    o = (1.0 - gamma) * np.asarray(g, np.float64) + gamma * gt
    o[fixed, 0], o[fixed, 1] = fx[fixed], fy[fixed]
    if clamp:
        xl, yl, xh, yh = region
        fr = ~fixed
        o[fr, 0] = np.minimum(np.maximum(o[fr, 0], xl + hw[fr]), xh - hw[fr])
        o[fr, 1] = np.minimum(np.maximum(o[fr, 1], yl + hh[fr]), yh - hh[fr])
    return o


def powers(o, gx, gy, kmax):
    """[g, H g, ..., H^kmax g] for an Oracle `o` whose hints are built, each
    power re-pinned when the parameters ask for it (as the plain filter)."""
    nd = o.nodes()
    fixed = nd["nkind"] == 2
    out = [np.stack([gx, gy], 1).astype(np.float64)]
    x, y = np.array(gx, np.float64), np.array(gy, np.float64)
    for _ in range(kmax):
        x, y = o.hr_steps(1, x), o.hr_steps(1, y)
        if o.params.pin_every_step:
            x[fixed], y[fixed] = nd["fx"][fixed], nd["fy"][fixed]
        out.append(np.stack([x, y], 1))
    return out


def round_inputs(o, gx, gy, k, rnd):
    """Everything the learned filter reads in one round, for an Oracle `o`
    whose hints are built at (gx, gy): taps G0, G1, G2 in bin units about the
    centre (powers k = (k0, k1, k2)), the raw features, and the scale and
    centre.  rnd: the round t of Algorithm 1 (feature 11 is t / T_hint)."""
    nd, sb, mg = o.nodes(), o.static_csr(), o.merged()
    nk = nd["nkind"]
    C, N = o.C, o.N
    xl, yl, xh, yh = o.nl.region
    s = np.array([(xh - xl) / o.params.nbx, (yh - yl) / o.params.nby])
    c = np.array([0.5 * (xl + xh), 0.5 * (yl + yh)])
    pw = powers(o, gx, gy, k[2])
    G0, G1, G2 = (bins(pw[kk], c, s) for kk in k)
    rp, w = mg["rp"], mg["w"]
    cs = np.concatenate([[0.0], np.cumsum(np.where(w > 0, w, 0.0))])
    psum = cs[rp[1:]] - cs[rp[:-1]]
    hint = np.zeros(N, bool)
    hint[:C] = (nk[:C] == 0) & (sb["base_w"] > 0)
    phi = np.zeros(N)
    if C:
        phi[:C] = np.where(hint[:C], mg["phi"][np.clip(mg["cell_bin"], 0, None)], 0.0)
    area = np.zeros(N)
    area[:C] = np.where(nk[:C] == 0, (2.0 * nd["hw"][:C]) * (2.0 * nd["hh"][:C]) / (s[0] * s[1]), 0.0)
    f = features(G0, G1, G2, mg["deg"], psum, mg["lam_up"], hint, phi, nk == 1, area,
                 rnd / o.params.t_hint)
    return dict(G0=G0, G1=G1, G2=G2, f=f, s=s, c=c, nkind=nk, free=nk != 2, nodes=nd)


def learned_round(o, gx, gy, k, rnd, w):
    """One round of Algorithm 1 with the learned filter in place of the plain
    one, for an Oracle whose hints are built at (gx, gy); w the parameter
    vector.  Returns (g' [N, 2], g~ [N, 2])."""
    r = round_inputs(o, gx, gy, k, rnd)
    p = unpack(w)
    _, _, out = mlp_forward(normalise(r["f"], p["mu"], p["isd"]), p)
    gt = r["c"] + r["s"] * predict(p["theta"], r["G0"], r["G1"], r["G2"], out)
    nd = r["nodes"]
    g1 = finish_round(gt, np.stack([gx, gy], 1), r["nkind"], nd["fx"], nd["fy"], nd["hw"],
                      nd["hh"], o.nl.region, o.params.gamma, o.params.clamp)
    return g1, gt
