"""Backward kernels (features and positions through IDW aggregation, the MLP
and Eq. 2) against the oracle's analytic backward, a directional finite
difference of the oracle's frozen forward on a 2k-point subset, and the
torch.autograd path."""
import numpy as np
import pytest
import torch

import oracle
from paper_2404_14044_b300 import scenes

pytestmark = pytest.mark.gpu


def _H():
    from paper_2404_14044_b300 import hashpoint
    return hashpoint


def _close(g, ref, rel=2e-4):
    scale = np.abs(ref).max()
    err = np.abs(g - ref).max()
    l2 = np.linalg.norm(g - ref) / max(np.linalg.norm(ref), 1e-30)
    assert err <= rel * scale and l2 <= rel, (err, scale, l2)
    return err / scale, l2


def _gpu_frame_grad(hp, pts_t, feats_t, cam, dims, mlp_t, rays_t, g_rgb_t, g_ws_t=None):
    H = _H()
    p = hp.params
    rgb, wsum, smp = hp.render(pts_t, feats_t, cam, dims, mlp_t, rays=rays_t)
    gf, gp = hp.aggregate_render_backward(smp, pts_t, feats_t, dims, mlp_t, g_rgb_t, g_ws_t)
    assert hp.status() == (0, 0)
    return rgb, wsum, smp, gf, gp


@pytest.mark.parametrize("mode,bg", [(scenes.RADIUS_FIXED, 0), (scenes.RADIUS_CONE_EXACT, 1)])
def test_backward_small_against_oracle(mode, bg):
    H = _H()
    dev = torch.device("cuda", 0)
    cam = scenes.make_camera(32, 32, 40.0, (0.0, -3.0, 0.0), t_near=1.0, t_far=10.0)
    pts = scenes.sphere_plane_points(4000, 4000, 1)
    feats = scenes.random_features(len(pts), 16, 2, std=0.5)
    p = scenes.Params(radius_mode=mode, r=0.04, rho=3.0 if mode else 0.0, K=6, n_max=6, bg_mode=bg, gamma=0.6)
    dims = [16, 32, 32, 4]
    mlp = scenes.random_mlp(dims, 3, sigma_bias=30.0)
    R = 32 * 32
    rng = np.random.default_rng(0)
    g_rgb = rng.normal(size=(R, 3)).astype(np.float32)
    g_ws = rng.normal(size=R).astype(np.float32)
    hp = H.HashPoint(p, dev)
    t = lambda a: torch.from_numpy(a).to(dev)
    rgb, wsum, smp, gf, gp = _gpu_frame_grad(hp, t(pts), t(feats), cam, dims, t(mlp), None, t(g_rgb), t(g_ws))
    fr = oracle.render(pts, feats, cam, p, dims, mlp, nthreads=8)
    of, _, opw = oracle.backward(pts, feats, cam, p, dims, mlp, fr, g_rgb.astype(np.float64), g_ws.astype(np.float64))
    _close(gf.cpu().numpy().astype(np.float64), of)
    _close(gp.cpu().numpy().astype(np.float64), opw)
    hp.close()


def test_training_step_four_views():
    # 4 views of the object scene, 4096 random rays each, MSE against an
    # oracle-rendered target made with a second feature draw
    H = _H()
    dev = torch.device("cuda", 0)
    n_pts = 1_000_000
    pts = scenes.object_points(n_pts, 0)
    feats = scenes.random_features(n_pts, 32, 1)
    feats_tgt = scenes.random_features(n_pts, 32, 7)
    p = scenes.Params(r=0.005, K=8, n_max=8)
    dims = [32, 128, 128, 128, 4]
    mlp = scenes.random_mlp(dims, 0, sigma_bias=1.5 / p.r)
    cams = scenes.random_sphere_cameras(4, 4.0, 0, width=800, height=800)
    t = lambda a: torch.from_numpy(a).to(dev)
    pts_t, feats_t, mlp_t = t(pts), t(feats), t(mlp)
    hp = H.HashPoint(p, dev)
    gf_gpu = torch.zeros_like(feats_t)
    gp_gpu = torch.zeros_like(pts_t)
    of = np.zeros((n_pts, 32))
    opw = np.zeros((n_pts, 3))
    frames = []
    rng = np.random.default_rng(0)
    total_n = 4 * 4096 * 3
    for v, cam in enumerate(cams):
        rays = np.sort(rng.choice(800 * 800, 4096, replace=False)).astype(np.int32)
        tgt = oracle.render(pts, feats_tgt, cam, p, dims, mlp, rays=rays, nthreads=8)["rgb"]
        rgb, wsum, smp = hp.render(pts_t, feats_t, cam, dims, mlp_t, rays=t(rays))
        g_rgb = (2.0 / total_n) * (rgb.double() - t(tgt)).float()
        hp.aggregate_render_backward(smp, pts_t, feats_t, dims, mlp_t, g_rgb, None, gf_gpu, gp_gpu)
        assert hp.status() == (0, 0)
        fr = oracle.render(pts, feats, cam, p, dims, mlp, rays=rays, nthreads=8)
        g_ref = (2.0 / total_n) * (fr["rgb"] - tgt)
        a, _, c = oracle.backward(pts, feats, cam, p, dims, mlp, fr, g_ref, None, rays=rays)
        of += a
        opw += c
        frames.append((cam, rays, fr, tgt))
    gfn, gpn = gf_gpu.cpu().numpy().astype(np.float64), gp_gpu.cpu().numpy().astype(np.float64)
    _close(gfn, of, rel=1e-3)
    _close(gpn, opw, rel=1e-3)
    assert (np.abs(of).sum(1) > 0).sum() > 10000

    # directional finite difference on a 2k-point subset (oracle frozen forward, FP64)
    touched = np.nonzero(np.abs(of).sum(1) > 0)[0]
    sub = rng.choice(touched, 2000, replace=False)
    vf = np.zeros_like(of)
    vf[sub] = rng.normal(size=(2000, 32))
    vp = np.zeros_like(opw)
    vp[sub] = rng.normal(size=(2000, 3))

    def loss(dfeat, dpos_world):
        L = 0.0
        for cam, rays, fr, tgt in frames:
            Rm = np.asarray(cam.R, np.float64).reshape(3, 3)
            pc0 = oracle.cam_points(cam, pts).astype(np.float64)
            pc = pc0 + dpos_world @ Rm.T
            rgb, _ = oracle.forward_frozen(pc, pc0, feats.astype(np.float64) + dfeat, cam, p, dims, mlp, fr, rays=rays)
            L += ((rgb - tgt) ** 2).sum() / total_n
        return L

    h = 1e-4
    fd_f = (loss(h * vf, 0 * vp) - loss(-h * vf, 0 * vp)) / (2 * h)
    assert abs(fd_f - (gfn * vf).sum()) <= 1e-3 * abs(fd_f) + 1e-9, (fd_f, (gfn * vf).sum())
    h = 1e-5
    fd_p = (loss(0 * vf, h * vp) - loss(0 * vf, -h * vp)) / (2 * h)
    assert abs(fd_p - (gpn * vp).sum()) <= 2e-3 * abs(fd_p) + 1e-9, (fd_p, (gpn * vp).sum())
    hp.close()


def test_autograd_function_matches_direct_call():
    H = _H()
    dev = torch.device("cuda", 0)
    sc = scenes.sphere_plane_64()
    t = lambda a: torch.from_numpy(a).to(dev)
    hp = H.HashPoint(sc.params, dev)
    feats = t(sc.feats).requires_grad_(True)
    pts = t(sc.points).requires_grad_(True)
    mlp = t(sc.mlp_params)
    rgb, wsum = H.render_differentiable(hp, feats, pts, sc.camera, sc.mlp_dims, mlp)
    loss = (rgb ** 2).sum() + 0.5 * wsum.sum()
    loss.backward()
    g_rgb = (2 * rgb).detach()
    g_ws = torch.full_like(wsum, 0.5)
    rgb2, wsum2, smp = hp.render(t(sc.points), t(sc.feats), sc.camera, sc.mlp_dims, mlp)
    gf, gp = hp.aggregate_render_backward(smp, t(sc.points), t(sc.feats), sc.mlp_dims, mlp, g_rgb, g_ws)
    assert torch.allclose(feats.grad, gf, rtol=1e-4, atol=1e-7)
    assert torch.allclose(pts.grad, gp, rtol=1e-4, atol=1e-6)
    assert feats.grad.abs().sum() > 0 and pts.grad.abs().sum() > 0
    hp.close()
