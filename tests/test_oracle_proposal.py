"""Pins of the proposal oracle (oracle/proposal.py) against facts fixed
outside it: points placed on known pixel rays at known depths, the closed
form of the interval map for a network with zero weights, central finite
differences of the loss, Adam's closed form at step 1, and torch's own
bfloat16 rounding."""
import numpy as np
import pytest
import torch

import oracle
from oracle import proposal as P
from paper_2404_14044_b300 import scenes


def _cam():
    return scenes.make_camera(32, 32, 40.0, (0.0, -4.0, 0.0), t_near=2.0, t_far=6.0)


def _point_on_pixel(cam, u, v, z):
    """World point whose camera-space position is depth z on the ray through
    the centre of pixel (u, v)."""
    Rm = np.asarray(cam.R, np.float64).reshape(3, 3)
    t = np.asarray(cam.t, np.float64)
    pc = np.array([z * (u + 0.5 - cam.cx) / cam.fx, z * (v + 0.5 - cam.cy) / cam.fy, z])
    return Rm.T @ (pc - t)


def test_bf16_round_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(size=5000) * 10.0 ** rng.integers(-6, 6, 5000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.0078125, 1.01171875]]).astype(np.float32)
    vals, bits = P.bf16_round(x)
    tb = torch.from_numpy(x).to(torch.bfloat16)
    assert np.array_equal(bits, tb.view(torch.int16).numpy().view(np.uint16))
    assert np.array_equal(vals, tb.double().numpy())


def test_counts_of_points_on_known_rays():
    cam = _cam()
    prm = scenes.Params(r=0.06)
    placed = [((10, 10), 2.1), ((10, 10), 2.2), ((10, 10), 5.9), ((11, 11), 3.1), ((13, 10), 4.1),
              ((9, 9), 7.5), ((9, 10), 1.0), ((-1, 10), 3.1)]
    pts = np.array([_point_on_pixel(cam, u, v, z) for (u, v), z in placed], np.float32)
    tab = oracle.build_table(pts, cam, prm)
    assert tab["h"] >= 1 and tab["n_visible"] == len(pts)
    px = lambda u, v: v * cam.width + u
    n = P.counts(tab, cam, [px(10, 10), px(12, 10), px(20, 20), px(0, 10), px(0, 0)])
    want = np.zeros((5, 16), np.int64)
    want[0, 0] = 3        # 2.1, 2.2 and 1.0 (before t_near: first bin)
    want[0, 4] = 1        # 3.1 at (11, 11)
    want[0, 15] = 2       # 5.9 and 7.5 (behind t_far: last bin)
    want[1, 4] = 1        # (11, 11)
    want[1, 8] = 1        # 4.1 at (13, 10)
    want[3, 4] = 1        # off-screen point at (-1, 10), inside the padded table
    assert np.array_equal(n, want)


def test_bin_index_float32_edges():
    # 16 bins over [2, 6]: width 0.25; float32 arithmetic at the exact edges
    z = np.array([2.0, 2.25, 2.2499998, 5.9999995, 6.0, 100.0, -1.0], np.float32)
    assert P.bin_index(z, 2.0, 6.0).tolist() == [0, 1, 0, 15, 15, 15, 0]


def test_intervals_closed_form_zero_weights():
    cam = _cam()
    th = np.zeros(P.N_PARAMS)
    th[-2:] = (0.7, -1.3)
    n = np.zeros((3, 16), np.int64)
    n[0, 3] = 5
    n[1, :] = 1
    iv = P.intervals(th, n, cam)
    s = lambda x: 1.0 / (1.0 + np.exp(-x))
    t0 = 2.0 + 4.0 * s(0.7)
    t1 = t0 + (6.0 - t0) * s(-1.3)
    assert np.allclose(iv[0], (t0, t1), rtol=0, atol=1e-14)
    assert np.allclose(iv[1], (t0, t1), rtol=0, atol=1e-14)
    assert tuple(iv[2]) == (2.0, 6.0)          # no point around the pixel: plain range


def test_forward_against_explicit_layers():
    th = scenes.proposal_params(3).astype(np.float64)
    rng = np.random.default_rng(1)
    x = np.log1p(rng.integers(0, 20, (7, 16)).astype(np.float64))
    o, _ = P.forward(th, x)
    # the packed layout written out by hand: W0 rows are outputs
    k = 0
    W0 = th[k:k + 512].reshape(32, 16); k += 512
    b0 = th[k:k + 32]; k += 32
    W1 = th[k:k + 1024].reshape(32, 32); k += 1024
    b1 = th[k:k + 32]; k += 32
    W2 = th[k:k + 64].reshape(2, 32); k += 64
    b2 = th[k:k + 2]
    for r in range(7):
        h1 = [max(sum(W0[j, i] * x[r, i] for i in range(16)) + b0[j], 0.0) for j in range(32)]
        h2 = [max(sum(W1[j, i] * h1[i] for i in range(32)) + b1[j], 0.0) for j in range(32)]
        for c in range(2):
            ref = sum(W2[c, i] * h2[i] for i in range(32)) + b2[c]
            assert abs(o[r, c] - ref) <= 1e-12 * (1 + abs(ref))


@pytest.mark.parametrize("seed", [0, 1])
def test_loss_gradient_finite_differences(seed):
    cam = _cam()
    rng = np.random.default_rng(seed)
    th = scenes.proposal_params(seed, out_bias=(0.0, 0.0), scale=0.5).astype(np.float64)
    R = 40
    n = rng.integers(0, 6, (R, 16))
    s0 = rng.uniform(2.2, 4.0, R)
    s1 = s0 + rng.uniform(0.0, 1.5, R)
    L, g, _ = P.loss_and_grad(th, n, s0, s1, cam)
    idx = rng.choice(P.N_PARAMS, 80, replace=False)
    idx = np.concatenate([idx, np.arange(P.N_PARAMS - 66, P.N_PARAMS)])   # all of W2, b2
    h = 1e-6
    for i in idx:
        e = np.zeros(P.N_PARAMS)
        e[i] = h
        fd = (P.loss_and_grad(th + e, n, s0, s1, cam)[0] - P.loss_and_grad(th - e, n, s0, s1, cam)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g).max()), (i, fd, g[i])
    d = rng.normal(size=P.N_PARAMS)
    fd = (P.loss_and_grad(th + h * d, n, s0, s1, cam)[0] - P.loss_and_grad(th - h * d, n, s0, s1, cam)[0]) / (2 * h)
    assert abs(fd - g @ d) <= 1e-6 * max(1.0, abs(fd))


def test_loss_pushes_interval_towards_the_samples():
    # zero weights: t0 and t1 come from b2 alone; an interval that starts
    # behind the first sample must get a gradient that lowers t0
    cam = _cam()
    th = np.zeros(P.N_PARAMS)
    th[-2:] = (0.0, 0.0)                 # t0 = 4, t1 = 5
    n = np.ones((1, 16), np.int64)
    _, g, _ = P.loss_and_grad(th, n, [3.0], [3.5], cam)
    assert g[-2] > 0                      # d L / d o0 > 0: descent lowers o0 (and t0)
    _, g, _ = P.loss_and_grad(th, n, [4.5], [5.8], cam)
    assert g[-1] < 0                      # last sample behind t1: descent raises o1


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(2)
    th = rng.normal(size=50)
    g = rng.normal(size=50)
    out, m, v = P.adam(th, np.zeros(50), np.zeros(50), g, 1, 1e-2)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 1e-3 * g * g)
    assert np.allclose(out, th - 1e-2 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
