"""Oracle of the learned depth-interval proposal -- test infrastructure.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU leg may
use this module.  It shares no code with the CUDA path; it takes the table
(bucket starts and camera-space positions) from the oracle's own
``build_table``.

The paper does not define this component.  It extends the method towards the
learned ray samplers that the paper lists as related work (Sec. 2), feeding
them from the hash table of Sec. 3.2.  The definition both sides implement:

* input      for the ray of pixel (u, v): n_b = the number of table points in
             the 3 x 3 buckets around the pixel (padded keys, clipped to the
             padded grid) whose camera depth z falls in bin
             b = clamp(floor((z - t_near) * (16 / (t_far - t_near))), 0, 15);
             the bin index is a discrete decision and is taken in float32
             (subtract, divide, multiply, each rounded once).  x_b = log(1 + n_b).
* network    16 -> 32 -> 32 -> 2, ReLU after the two hidden layers.
* interval   t0 = t_near + (t_far - t_near) sigmoid(o0),
             t1 = t0 + (t_far - t0) sigmoid(o1).  A ray with no point around
             its pixel gets [t_near, t_far] (the plain search).  Inference
             uses the weights rounded to bfloat16 (round to nearest even).
* loss       per ray with at least one plain-search sample (first depth s0,
             last s1), depths in units of the range, u(t) = (t - t_near) /
             (t_far - t_near):
             softplus(k (u(t0) - u(s0) + m)) / k + softplus(k (u(s1) - u(t1) + m)) / k
             + lam (u(t1) - u(t0)),   k = 200, m = 0.01, lam = 0.05.
             The training gradient is the mean over those rays.
* update     Adam (Kingma & Ba, ICLR 2015): beta1 = 0.9, beta2 = 0.999,
             eps = 1e-8, bias-corrected.

Parameter vector (1666 float32): W0 (32 x 16, row-major: output-major), b0
(32), W1 (32 x 32), b1 (32), W2 (2 x 32), b2 (2).  Continuous values are
float64.  Pins (tests/test_oracle_proposal.py): histograms against points
placed on known rays at known depths, the interval map's closed form for a
network with zero weights, the loss gradient against central finite
differences, Adam against its closed form at step 1.
"""
from __future__ import annotations

import numpy as np

BINS, HID = 16, 32
N_PARAMS = HID * BINS + HID + HID * HID + HID + 2 * HID + 2
KAPPA, MARGIN, LAMBDA = 200.0, 0.01, 0.05


def unpack(theta):
    """Split the parameter vector into (W0, b0, W1, b1, W2, b2), float64."""
    th = np.asarray(theta, np.float64).reshape(-1)
    assert th.size == N_PARAMS
    o = 0
    out = []
    for shape in [(HID, BINS), (HID,), (HID, HID), (HID,), (2, HID), (2,)]:
        n = int(np.prod(shape))
        out.append(th[o:o + n].reshape(shape))
        o += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(p, np.float64).reshape(-1) for p in parts])


def bf16_round(theta_f32):
    """bfloat16 rounding (nearest, ties to even) of float32 values: returns
    (the rounded values as float64, their 16-bit patterns)."""
    u = np.ascontiguousarray(theta_f32, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16
    bits = u.astype(np.uint16)
    vals = (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    return vals, bits


def bin_index(z, t_near, t_far):
    """Depth bin of float32 depths, in float32 arithmetic."""
    z = np.asarray(z, np.float32)
    tn, tf = np.float32(t_near), np.float32(t_far)
    scale = np.float32(BINS) / np.float32(tf - tn)
    v = np.floor((z - tn) * scale)
    return np.clip(v, 0, BINS - 1).astype(np.int64)


def counts(table, cam, pixels):
    """n_b per ray (R x 16 int64) from the oracle table (``build_table``)."""
    h = table["h"]
    Wp, Hp = cam.width + 2 * h, cam.height + 2 * h
    start = table["start"].astype(np.int64)
    z = table["pos"][:, 2] if table["n_visible"] > 0 else np.zeros(0, np.float32)
    pix = np.asarray(pixels, np.int64)
    R = len(pix)
    n = np.zeros((R, BINS), np.int64)
    pu, pv = pix % cam.width, pix // cam.width
    c0 = np.maximum(pu + h - 1, 0)
    c1 = np.minimum(pu + h + 1, Wp - 1)
    for dr in (-1, 0, 1):
        row = pv + h + dr
        ok = (row >= 0) & (row < Hp)
        lo = np.where(ok, start[np.clip(row, 0, Hp - 1) * Wp + c0], 0)
        hi = np.where(ok, start[np.clip(row, 0, Hp - 1) * Wp + c1 + 1], 0)
        ln = hi - lo
        ray = np.repeat(np.arange(R), ln)
        idx = np.repeat(lo - np.concatenate([[0], np.cumsum(ln)[:-1]]), ln) + np.arange(ln.sum())
        if idx.size:
            np.add.at(n, (ray, bin_index(z[idx], cam.t_near, cam.t_far)), 1)
    return n


def features(n):
    return np.log1p(np.asarray(n, np.float64))


def forward(theta, x):
    """Network outputs (R x 2) and the hidden activations."""
    W0, b0, W1, b1, W2, b2 = unpack(theta)
    z1 = x @ W0.T + b0
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W1.T + b1
    h2 = np.maximum(z2, 0.0)
    o = h2 @ W2.T + b2
    return o, (z1, h1, z2, h2)


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def intervals(theta, n, cam):
    """[t0, t1] per ray (R x 2, float64) from the counts n (R x 16)."""
    o, _ = forward(theta, features(n))
    tn, tf = float(np.float32(cam.t_near)), float(np.float32(cam.t_far))
    t0 = tn + (tf - tn) * sigmoid(o[:, 0])
    t1 = t0 + (tf - t0) * sigmoid(o[:, 1])
    out = np.stack([t0, t1], 1)
    out[n.sum(1) == 0] = (tn, tf)
    return out


def softplus(x):
    return np.log1p(np.exp(-np.abs(x))) + np.maximum(x, 0.0)


def loss_and_grad(theta, n, s0, s1, cam):
    """Mean loss and its gradient w.r.t. the parameter vector over the rays
    given (each with a first / last plain-search sample depth s0, s1)."""
    x = features(n)
    W0, b0, W1, b1, W2, b2 = unpack(theta)
    o, (z1, h1, z2, h2) = forward(theta, x)
    tn, tf = float(np.float32(cam.t_near)), float(np.float32(cam.t_far))
    span = tf - tn
    u0, u1 = sigmoid(o[:, 0]), sigmoid(o[:, 1])
    t0n = u0
    t1n = u0 + (1.0 - u0) * u1
    s0n = (np.asarray(s0, np.float64) - tn) / span
    s1n = (np.asarray(s1, np.float64) - tn) / span
    e0 = KAPPA * (t0n - s0n + MARGIN)
    e1 = KAPPA * (s1n - t1n + MARGIN)
    R = len(x)
    loss = (softplus(e0) + softplus(e1)) / KAPPA + LAMBDA * (t1n - t0n)
    # chain rule, per ray, then the mean
    g_t0n = sigmoid(e0) - LAMBDA
    g_t1n = -sigmoid(e1) + LAMBDA
    g_u0 = g_t0n + g_t1n * (1.0 - u1)
    g_u1 = g_t1n * (1.0 - u0)
    g_o = np.stack([g_u0 * u0 * (1.0 - u0), g_u1 * u1 * (1.0 - u1)], 1) / R
    gW2 = g_o.T @ h2
    gb2 = g_o.sum(0)
    g_z2 = (g_o @ W2) * (z2 > 0)
    gW1 = g_z2.T @ h1
    gb1 = g_z2.sum(0)
    g_z1 = (g_z2 @ W1) * (z1 > 0)
    gW0 = g_z1.T @ x
    gb0 = g_z1.sum(0)
    return float(loss.mean()), pack([gW0, gb0, gW1, gb1, gW2, gb2]), float(loss.sum())


def adam(theta, m, v, g, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step; returns (theta, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def plain_targets(frame):
    """(ray index, s0, s1) of the rays with samples in an oracle frame."""
    ns = frame["n_s"]
    off = frame["sample_offset"]
    hit = np.nonzero(ns > 0)[0]
    t = frame["t"].astype(np.float64)
    return hit, t[off[hit]], t[off[hit] + ns[hit] - 1]
