"""Learned depth-interval proposal: training/inference kernels, the
interval-restricted search with plain fallback (bit-exact against the
oracle given the same intervals), and its miss rate judged by the plain
search."""
import numpy as np
import pytest
import torch

import oracle
from paper_2404_14044_b300 import scenes
from tests.test_gpu_parity import assert_parity

pytestmark = pytest.mark.gpu


def _H():
    from paper_2404_14044_b300 import hashpoint
    return hashpoint


def _frame(hp, pts_t, feats_t, cam, dims, mlp_t, interval=None):
    p = hp.params
    hp.build_table(pts_t, cam, p.r)
    if interval is None:
        smp = hp.search_sample(None, p.K, p.n_max)
    else:
        smp = hp.search_sample_proposal(None, p.K, p.n_max, interval)
    rgb, wsum = hp.aggregate_render(smp, feats_t, dims, mlp_t)
    st = hp.status()
    R = cam.width * cam.height
    out = smp.packed(R)
    out = {k: (v.numpy() if isinstance(v, torch.Tensor) else v) for k, v in out.items()}
    out["rgb"] = rgb.cpu().numpy().astype(np.float64)
    out["wsum"] = wsum.cpu().numpy().astype(np.float64)
    out["status"] = st
    return out


def test_full_interval_equals_plain():
    H = _H()
    dev = torch.device("cuda", 0)
    sc = scenes.objects_800(n_points=300_000, res=200)
    t = lambda a: torch.from_numpy(a).to(dev)
    hp = H.HashPoint(sc.params, dev)
    R = 200 * 200
    full = torch.tensor([[sc.camera.t_near, sc.camera.t_far]], device=dev).repeat(R, 1).contiguous()
    a = _frame(hp, t(sc.points), t(sc.feats), sc.camera, sc.mlp_dims, t(sc.mlp_params))
    b = _frame(hp, t(sc.points), t(sc.feats), sc.camera, sc.mlp_dims, t(sc.mlp_params), interval=full)
    for k in ("n_s", "primary", "cand_count", "t", "src", "nbr", "nbr_dist", "rgb"):
        assert np.array_equal(a[k], b[k]), k
    hp.close()


def test_train_infer_and_restricted_parity():
    H = _H()
    dev = torch.device("cuda", 0)
    res = 256
    pts = scenes.object_points(1_000_000, 0)
    feats = scenes.random_features(len(pts), 32, 1)
    p = scenes.Params(r=0.005, K=8, n_max=8)
    dims = [32, 128, 128, 128, 4]
    mlp = scenes.random_mlp(dims, 0, sigma_bias=1.5 / p.r)
    cams = scenes.random_sphere_cameras(17, 4.0, 3, width=res, height=res)
    t = lambda a: torch.from_numpy(a).to(dev)
    pts_t, feats_t, mlp_t = t(pts), t(feats), t(mlp)
    hp = H.HashPoint(p, dev)
    state = H.ProposalState(dev, seed=0)
    losses = []
    for step in range(240):
        cam = cams[step % 16]
        hp.build_table(pts_t, cam, p.r)
        plain = hp.search_sample(None, p.K, p.n_max)
        hp.proposal_train_step(None, plain, state, lr=3e-3)
        if step % 16 == 15:
            l = state.loss.cpu().numpy()
            losses.append(l[0] / max(l[1], 1))
    assert hp.status() == (0, 0)
    assert losses[-1] < 0.5 * losses[0], losses
    # held-out view: infer, restricted search, compare with the oracle (same intervals) and with plain
    cam = cams[16]
    hp.build_table(pts_t, cam, p.r)
    iv = hp.proposal_infer(None, state.bf16)
    g = _frame(hp, pts_t, feats_t, cam, dims, mlp_t, interval=iv)
    ivn = iv.cpu().numpy()
    o = oracle.render(pts, feats, cam, p, dims, mlp, nthreads=8, intervals=ivn)
    assert_parity(g, o, p.K)
    plain = _frame(hp, pts_t, feats_t, cam, dims, mlp_t)
    assert np.all((g["n_s"] == 0) <= (plain["n_s"] == 0))          # empty only where plain is empty
    hit = plain["n_s"] > 0
    same = np.array([np.array_equal(g["src"][g["sample_offset"][i]:g["sample_offset"][i + 1]],
                                    plain["src"][plain["sample_offset"][i]:plain["sample_offset"][i + 1]])
                     for i in np.nonzero(hit)[0]])
    miss = 1.0 - same.mean()
    print(f"proposal miss rate {miss:.4f} on {hit.sum()} hit rays; losses {losses[0]:.4f} -> {losses[-1]:.4f}")
    assert miss < 0.10
    hp.close()
