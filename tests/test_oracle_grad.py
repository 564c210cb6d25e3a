"""Pins of the oracle's analytic backward (features and positions through
IDW aggregation, the MLP and Eq. 2 compositing, discrete structure frozen):
central finite differences of the frozen forward, and consistency of the
frozen forward with the regular forward at the base point.  CPU only."""
import numpy as np
import pytest

import oracle
from paper_2404_14044_b300 import scenes


def _setup(mode=scenes.RADIUS_FIXED, bg=0, gamma=0.9, seed=0):
    cam = scenes.make_camera(24, 24, 40.0, (0.0, -3.0, 0.0), t_near=1.0, t_far=10.0)
    pts = scenes.sphere_plane_points(3000, 3000, seed)
    feats = scenes.random_features(len(pts), 8, seed + 1, std=0.5)
    p = scenes.Params(radius_mode=mode, r=0.05, rho=3.0 if mode else 0.0, K=4, n_max=4, bg_mode=bg, gamma=gamma)
    dims = [8, 16, 16, 4]
    mlp = scenes.random_mlp(dims, seed, sigma_bias=20.0)
    fr = oracle.render(pts, feats, cam, p, dims, mlp)
    return cam, pts, feats, p, dims, mlp, fr


def test_frozen_forward_matches_forward_at_base():
    cam, pts, feats, p, dims, mlp, fr = _setup()
    pc = oracle.cam_points(cam, pts).astype(np.float64)
    rgb, ws = oracle.forward_frozen(pc, pc, feats.astype(np.float64), cam, p, dims, mlp, fr)
    assert np.allclose(rgb, fr["rgb"], rtol=1e-12, atol=1e-14) and np.allclose(ws, fr["wsum"], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("mode,bg,gamma", [(scenes.RADIUS_FIXED, 0, 0.9), (scenes.RADIUS_CONE_EXACT, 1, 0.5),
                                          (scenes.RADIUS_FIXED, 1, 0.3)])
def test_backward_against_finite_differences(mode, bg, gamma):
    cam, pts, feats, p, dims, mlp, fr = _setup(mode, bg, gamma)
    R = len(fr["n_s"])
    rng = np.random.default_rng(5)
    g_rgb = rng.normal(size=(R, 3))
    g_ws = rng.normal(size=R)
    gf, gpc, gpw = oracle.backward(pts, feats, cam, p, dims, mlp, fr, g_rgb, g_ws)
    pc0 = oracle.cam_points(cam, pts).astype(np.float64)
    f0 = feats.astype(np.float64)

    def loss(pc, f):
        rgb, ws = oracle.forward_frozen(pc, pc0, f, cam, p, dims, mlp, fr)
        return float((rgb * g_rgb).sum() + (ws * g_ws).sum())

    used = np.unique(np.concatenate([fr["src"], fr["nbr"][fr["nbr"] >= 0]]))
    assert len(used) > 50
    pick = rng.choice(used, 25, replace=False)
    h = 1e-6
    for i in pick:
        for k in rng.choice(feats.shape[1], 3, replace=False):
            fp, fm = f0.copy(), f0.copy()
            fp[i, k] += h
            fm[i, k] -= h
            fd = (loss(pc0, fp) - loss(pc0, fm)) / (2 * h)
            assert abs(fd - gf[i, k]) <= 1e-5 * max(1.0, abs(fd)), (i, k, fd, gf[i, k])
        for a in range(3):
            pp, pm = pc0.copy(), pc0.copy()
            pp[i, a] += h
            pm[i, a] -= h
            fd = (loss(pp, f0) - loss(pm, f0)) / (2 * h)
            assert abs(fd - gpc[i, a]) <= 1e-4 * max(1.0, abs(fd)), (i, a, fd, gpc[i, a])
    # world-space gradient is R^T times the camera-space one
    Rm = np.asarray(cam.R, np.float64).reshape(3, 3)
    assert np.allclose(gpw, gpc @ Rm, rtol=1e-12, atol=1e-12)
    # points that no sample touches get no gradient
    unused = np.setdiff1d(np.arange(len(pts)), used)
    assert np.all(gf[unused] == 0) and np.all(gpc[unused] == 0)
