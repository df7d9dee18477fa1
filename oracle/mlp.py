"""Oracle of the learned skin network (8 -> 32 -> 32 -> 1, ReLU).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper sets each particle's skin by the rule skin = K |v| dt (Eq.
skin_formulus1).  The learned variant replaces the rule by a small network
that reads eight features of the particle's local kinematics and proposes a
skin; the displacement check of Eq. update still guards every list, so a
poor proposal costs time, never a missed contact.  The paper gives no
network, so everything below is this project's reading.

Inference formula (exact: any implementation evaluating it gets the same
bits):
    z_k  = bf16( (f_k - mu_k) * isd_k )               binary32, then RN-even
    h1_o = bf16( relu( b1_o + sum_k W1_ok z_k ) )      k = 0..7 in order
    h2_o = bf16( relu( b2_o + sum_k W2_ok h1_k ) )     k = 0..31 in order
    y    = b3 + sum_k w3_k h2_k                        k = 0..31 in order
    yc   = fmin(fmax(y, y_lo), y_hi)
    skin = d * yc                          diameter form (y_steps = 0)
    skin = d * (f0 * (yc * y_steps))       travel form (y_steps > 0)
(each product one binary32 rounding, in that order; then the cap; fmax /
fmin return the other operand when one is NaN.)  The output range
[y_lo, y_hi] and y_steps belong to the weights; y_lo = 0, y_hi = +inf gives
yc = max(y, 0).  Since f0 d is the particle's travel |v| dt in one step,
the travel form is the paper's rule K |v| dt with a per-particle factor
K = yc * y_steps proposed by the network.
Weights and biases are bfloat16 / binary32; each product of two bfloat16
values is exact in binary32, and each sum is one binary32 rounding, taken
in the order written, starting from the bias.

Training reference (binary64): the same network with the bfloat16
roundings of z, h1, h2 and of the weights applied in the forward pass and
treated as the identity in the backward pass (straight-through), loss =
mean squared error of y against the label.
"""
from __future__ import annotations

import numpy as np

N_IN, N_H = 8, 32
N_PARAMS = N_H * N_IN + N_H + N_H * N_H + N_H + N_H + 1   # 1,377


def bf16_round(x):
    """binary32 -> bfloat16 (round to nearest, ties to even), returned as
    binary32 values.  NaN stays NaN."""
    a = np.ascontiguousarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) & 0xFFFF0000).astype(np.uint32)
    out = r.view(np.float32).copy()
    nan = np.isnan(a)
    out[nan] = np.nan
    return out.reshape(np.shape(x))


class Weights:
    """Parameters in binary32 master form."""

    def __init__(self, W1, b1, W2, b2, w3, b3, mu, isd, y_lo=0.0, y_hi=np.inf, y_steps=0.0):
        self.W1 = np.asarray(W1, np.float32).reshape(N_H, N_IN)
        self.b1 = np.asarray(b1, np.float32).reshape(N_H)
        self.W2 = np.asarray(W2, np.float32).reshape(N_H, N_H)
        self.b2 = np.asarray(b2, np.float32).reshape(N_H)
        self.w3 = np.asarray(w3, np.float32).reshape(N_H)
        self.b3 = np.float32(b3)
        self.mu = np.asarray(mu, np.float32).reshape(N_IN)
        self.isd = np.asarray(isd, np.float32).reshape(N_IN)
        self.y_lo = np.float32(y_lo)
        self.y_hi = np.float32(y_hi)
        self.y_steps = np.float32(y_steps)

    @staticmethod
    def random(seed=0, scale=0.3):
        rng = np.random.default_rng(seed)
        return Weights(rng.normal(0, scale, (N_H, N_IN)), rng.normal(0, 0.1, N_H),
                       rng.normal(0, scale / 3, (N_H, N_H)), rng.normal(0, 0.1, N_H),
                       rng.normal(0, scale / 3, N_H), 0.05, np.zeros(N_IN), np.ones(N_IN))

    def flat(self):
        return np.concatenate([self.W1.ravel(), self.b1, self.W2.ravel(), self.b2, self.w3,
                               [self.b3]]).astype(np.float32)

    @staticmethod
    def from_flat(p, mu, isd, y_lo=0.0, y_hi=np.inf, y_steps=0.0):
        p = np.asarray(p, np.float32)
        o = 0
        W1 = p[o:o + N_H * N_IN]; o += N_H * N_IN
        b1 = p[o:o + N_H]; o += N_H
        W2 = p[o:o + N_H * N_H]; o += N_H * N_H
        b2 = p[o:o + N_H]; o += N_H
        w3 = p[o:o + N_H]; o += N_H
        b3 = p[o]
        return Weights(W1, b1, W2, b2, w3, b3, mu, isd, y_lo, y_hi, y_steps)


def _dot_fixed(bias, w, x):
    """bias + sum_k w_k x_k in binary32, k in order, rows of w in parallel.
    w: (O, K) bf16 values as float32, x: (..., K); products are exact."""
    acc = np.broadcast_to(np.float32(0), x.shape[:-1] + (w.shape[0],)).astype(np.float32)
    acc = acc + bias.astype(np.float32)
    for k in range(w.shape[1]):
        prod = (w[:, k][None, :].astype(np.float64) * x[..., k:k + 1].astype(np.float64))
        prod = prod.astype(np.float32)               # exact for bf16 x bf16
        acc = (acc + prod).astype(np.float32)
    return acc


def infer(W: Weights, feats, diam):
    """The exact inference formula: skin proposal per row of feats (n, 8)."""
    f = np.asarray(feats, np.float32).reshape(-1, N_IN)
    z = bf16_round(((f - W.mu).astype(np.float32) * W.isd).astype(np.float32))
    h1 = bf16_round(np.maximum(_dot_fixed(W.b1, bf16_round(W.W1), z), np.float32(0)))
    h2 = bf16_round(np.maximum(_dot_fixed(W.b2, bf16_round(W.W2), h1), np.float32(0)))
    y = _dot_fixed(np.array([W.b3], np.float32), bf16_round(W.w3)[None, :], h2)[:, 0]
    yc = np.fmin(np.fmax(y, W.y_lo), W.y_hi).astype(np.float32)
    if W.y_steps > 0:
        k = (yc * W.y_steps).astype(np.float32)
        yc = (f[:, 0] * k).astype(np.float32)
    return (np.asarray(diam, np.float32) * yc).astype(np.float32), y


def forward64(W: Weights, feats, quantize=True):
    """binary64 forward with the bfloat16 roundings of the inference path
    (none when quantize is False).  Returns (y, cache)."""
    q = bf16_round if quantize else (lambda a: np.asarray(a))
    f = np.asarray(feats, np.float64 if not quantize else np.float32).reshape(-1, N_IN)
    if quantize:
        z = q(((f - W.mu).astype(np.float32) * W.isd).astype(np.float32)).astype(np.float64)
    else:
        z = (f - W.mu.astype(np.float64)) * W.isd.astype(np.float64)
    W1 = np.asarray(q(W.W1), np.float64)
    W2 = np.asarray(q(W.W2), np.float64)
    w3 = np.asarray(q(W.w3), np.float64)
    a1 = z @ W1.T + W.b1.astype(np.float64)
    h1 = np.maximum(a1, 0)
    if quantize:
        h1 = q(h1.astype(np.float32)).astype(np.float64)
    a2 = h1 @ W2.T + W.b2.astype(np.float64)
    h2 = np.maximum(a2, 0)
    if quantize:
        h2 = q(h2.astype(np.float32)).astype(np.float64)
    y = h2 @ w3 + float(W.b3)
    return y, (z, a1, h1, a2, h2, W2, w3)


def loss_and_grad64(W: Weights, feats, labels, quantize=True, rel_floor=0.0):
    """Mean squared error and its gradient with respect to the flat
    parameters (order of Weights.flat), binary64; with quantize the bfloat16
    roundings act in the forward pass and as the identity backwards.  With
    rel_floor > 0 the error of each sample is relative to its label (not
    below rel_floor): mean of ((y - t) / max(t, rel_floor))^2."""
    y, (z, a1, h1, a2, h2, W2, w3) = forward64(W, feats, quantize)
    t = np.asarray(labels, np.float64).reshape(-1)
    B = len(t)
    r = y - t
    if rel_floor > 0.0:
        w = 1.0 / np.maximum(t, float(np.float32(rel_floor))) ** 2
    else:
        w = np.ones_like(t)
    loss = float(np.mean(w * r * r))
    dy = 2.0 * w * r / B
    gw3 = h2.T @ dy
    gb3 = dy.sum()
    dh2 = np.outer(dy, w3) * (a2 > 0)
    gW2 = dh2.T @ h1
    gb2 = dh2.sum(axis=0)
    dh1 = (dh2 @ W2) * (a1 > 0)
    gW1 = dh1.T @ z
    gb1 = dh1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, [gb3]])
    return loss, g


# ----------------------------------------------------------------- features
def _f32(x):
    return np.asarray(x, dtype=np.float32)


def _norm3(a):
    """sqrt((x*x + y*y) + z*z), binary32, correctly rounded square root."""
    a = _f32(a)
    s = (a[:, 0] * a[:, 0] + a[:, 1] * a[:, 1]).astype(np.float32)
    s = (s + a[:, 2] * a[:, 2]).astype(np.float32)
    return np.sqrt(s).astype(np.float32)


def grid_params(rmax, cell_factor, lo, hi):
    """The cell grid the features refer to: edge L = cell_factor * 2 rmax *
    (1 + 2^-7) (widened so that no axis needs more than 2048 cells), cells
    per axis ceil(extent / L) clamped to [1, 2048], invL = 1/L rounded to
    binary32, and the cap H = L/2 (1 - 2^-8) rounded to binary32."""
    L = float(cell_factor) * 2.0 * float(np.float32(rmax)) * (1.0 + 2.0 ** -7)
    ext = max(float(np.float32(h)) - float(np.float32(l)) for l, h in zip(lo, hi))
    if ext / L > 2048.0:
        L = ext / 2048.0
    dims = [int(min(max(np.ceil((float(np.float32(h)) - float(np.float32(l))) / L), 1), 2048))
            for l, h in zip(lo, hi)]
    return {"lo": _f32(lo), "hi": _f32(hi), "invL": np.float32(1.0 / L), "dims": dims,
            "H": np.float32(0.5 * L * (1.0 - 2.0 ** -8))}


def cell_index(x, grid):
    """Cell of each point: floor((x - lo) * invL) in binary32, clamped."""
    x = _f32(x)
    key = np.zeros(len(x), dtype=np.int64)
    mul = 1
    for k in range(3):
        u = ((x[:, k] - grid["lo"][k]).astype(np.float32) * grid["invL"]).astype(np.float32)
        u = np.clip(u, -1.0, grid["dims"][k]).astype(np.float32)
        c = np.clip(np.floor(u).astype(np.int64), 0, grid["dims"][k] - 1)
        key += c * mul
        mul *= grid["dims"][k]
    return key


def features(pos4, vel4, acc4, dt, grid, ref_old, nrow, age, occ):
    """The eight features of lvb_mlp.h for the given particles (binary32).
    pos4: (m, 4) x, y, z, r; vel4/acc4: (m, 4); ref_old: (m, 4) old
    reference state; nrow, age, occ: (m,) integers."""
    pos4, vel4, acc4, ref_old = _f32(pos4), _f32(vel4), _f32(acc4), _f32(ref_old)
    dt = np.float32(dt)
    r = pos4[:, 3]
    d = (np.float32(2.0) * r).astype(np.float32)
    f = np.zeros((len(pos4), N_IN), dtype=np.float32)
    f[:, 0] = ((_norm3(vel4) * dt).astype(np.float32) / d).astype(np.float32)
    f[:, 1] = ((((_norm3(acc4) * dt).astype(np.float32)) * dt).astype(np.float32) / d)
    f[:, 2] = (r / grid["H"]).astype(np.float32)
    f[:, 3] = np.asarray(nrow, dtype=np.float32)
    f[:, 4] = np.asarray(age, dtype=np.float32)
    dx = (pos4[:, :3] - ref_old[:, :3]).astype(np.float32)
    dist = _norm3(dx)
    so = ref_old[:, 3]
    with np.errstate(divide="ignore", invalid="ignore"):
        f5 = (dist / so).astype(np.float32)
    f[:, 5] = np.where(so > 0, f5, np.float32(0))
    f[:, 6] = np.asarray(occ, dtype=np.float32)
    w = None
    for k in range(3):
        lo_gap = ((pos4[:, k] - grid["lo"][k]).astype(np.float32) - r).astype(np.float32)
        hi_gap = ((grid["hi"][k] - pos4[:, k]).astype(np.float32) - r).astype(np.float32)
        m = np.minimum(lo_gap, hi_gap)
        w = m if w is None else np.minimum(w, m)
    f[:, 7] = (w / d).astype(np.float32)
    return f


# ----------------------------------------------------------------- labels
def travel_labels(samples, horizon, margin, clip_q):
    """Rebuild-log samples (n, 9: eight features, label = largest
    displacement over the horizon / d) as training samples of the travel
    form over `horizon` steps.  In the order given, the samples with
    f0 > 0 are kept (f0 d = |v| dt is the particle's travel per step; one at
    rest has none); each label t becomes y = (t * margin) / (f0 * horizon),
    every operation rounded to binary32 -- the displacement in units of the
    travel over the horizon, times a margin -- and then y = min(y, c) with c
    the value of rank k = floor(clip_q (m - 1)) (0-based) among the m values
    y in ascending order."""
    s = np.asarray(samples, dtype=np.float32).reshape(-1, N_IN + 1)
    kept = s[s[:, 0] > np.float32(0)].copy()
    m = len(kept)
    if m == 0:
        return kept
    t = (kept[:, N_IN] * np.float32(margin)).astype(np.float32)
    u = (kept[:, 0] * np.float32(horizon)).astype(np.float32)
    y = (t / u).astype(np.float32)
    k = int(np.floor(float(np.float32(clip_q)) * float(m - 1)))
    c = np.sort(y)[k]
    kept[:, N_IN] = np.minimum(y, c)
    return kept
