"""Neighbour lists left in the search's workspace (hp_samples.nbr NULL): the
render reads them there and must give exactly the image of the packed lists
(same samples, same arithmetic), in every decode path; the backward refuses
them."""
import numpy as np
import pytest
import torch

from paper_2404_14044_b300 import scenes

pytestmark = pytest.mark.gpu


def _H():
    from paper_2404_14044_b300 import hashpoint
    return hashpoint


def _scene(which):
    if which == "sphere_plane_64":
        return scenes.sphere_plane_64()
    if which == "objects_200":
        return scenes.objects_800(n_points=250_000, res=200)
    if which == "sphere_plane_64_k3":
        sc = scenes.sphere_plane_64()
        sc.params.K = 3                       # K not a multiple of 4: plain list loads
        return sc
    if which == "forward_252":
        return scenes.forward_1008(n_field=200_000, n_occ=50_000, width=252, height=189)   # K = 16
    raise ValueError(which)


def _frame(hp, sc, dev, lists, decode):
    H = _H()
    R = sc.camera.width * sc.camera.height
    pts = torch.from_numpy(sc.points).to(dev)
    feats = torch.from_numpy(sc.feats).to(dev)
    mlp = torch.from_numpy(sc.mlp_params).to(dev)
    smp = H.SampleBuffers.allocate(R, sc.params.K, sc.params.n_max, dev, lists=lists)
    hp.build_table(pts, sc.camera, sc.params.r)
    hp.search_sample(None, sc.params.K, sc.params.n_max, out=smp)
    rgb, wsum = hp.aggregate_render(smp, feats, sc.mlp_dims, mlp, decode=decode)
    torch.cuda.synchronize()
    return rgb.clone(), wsum.clone(), smp


@pytest.mark.parametrize("which", ["sphere_plane_64", "objects_200", "sphere_plane_64_k3", "forward_252"])
def test_workspace_lists_render_identical(which):
    H = _H()
    dev = torch.device("cuda", 0)
    sc = _scene(which)
    hp = H.HashPoint(sc.params, dev)
    R = sc.camera.width * sc.camera.height
    for decode in (H.DECODE_FP32, H.DECODE_BF16, H.DECODE_FP32_SIMT):
        rgb_p, ws_p, smp_p = _frame(hp, sc, dev, True, decode)
        assert hp.status() == (0, 0)
        rgb_w, ws_w, smp_w = _frame(hp, sc, dev, False, decode)
        assert hp.status() == (0, 0)
        S = int(smp_p.sample_offset[R].item())
        assert S > 0 and S == int(smp_w.sample_offset[R].item())
        for f in ("n_s", "primary", "cand_count", "sample_offset"):
            assert torch.equal(getattr(smp_p, f), getattr(smp_w, f)), f
        for f in ("t", "ray", "src", "delta"):
            assert torch.equal(getattr(smp_p, f)[:S], getattr(smp_w, f)[:S]), f
        # bit-identical colours and weight sums
        assert torch.equal(rgb_p.view(torch.int32), rgb_w.view(torch.int32)), (which, decode)
        assert torch.equal(ws_p.view(torch.int32), ws_w.view(torch.int32)), (which, decode)
    hp.close()


def test_workspace_lists_rules():
    H = _H()
    dev = torch.device("cuda", 0)
    sc = scenes.sphere_plane_64()
    hp = H.HashPoint(sc.params, dev)
    R = sc.camera.width * sc.camera.height
    pts = torch.from_numpy(sc.points).to(dev)
    feats = torch.from_numpy(sc.feats).to(dev)
    mlp = torch.from_numpy(sc.mlp_params).to(dev)
    # lists in the workspace: the backward needs them packed
    rgb, wsum, smp = _frame(hp, sc, dev, False, H.DECODE_FP32)
    with pytest.raises(RuntimeError):
        hp.aggregate_render_backward(smp, pts, feats, sc.mlp_dims, mlp, torch.ones_like(rgb))
    # a packed search, then a render asking for workspace lists
    smp_p = H.SampleBuffers.allocate(R, sc.params.K, sc.params.n_max, dev, lists=True)
    hp.build_table(pts, sc.camera, sc.params.r)
    hp.search_sample(None, sc.params.K, sc.params.n_max, out=smp_p)
    smp_w = H.SampleBuffers.allocate(R, sc.params.K, sc.params.n_max, dev, lists=False)
    smp_w.n_s, smp_w.primary, smp_w.cand_count = smp_p.n_s, smp_p.primary, smp_p.cand_count
    smp_w.sample_offset, smp_w.t, smp_w.ray, smp_w.src, smp_w.delta = (smp_p.sample_offset, smp_p.t, smp_p.ray,
                                                                      smp_p.src, smp_p.delta)
    with pytest.raises(RuntimeError):
        hp.aggregate_render(smp_w, feats, sc.mlp_dims, mlp)
    # one list pointer without the other
    smp_p.nbr_dist = None
    with pytest.raises(RuntimeError):
        hp.search_sample(None, sc.params.K, sc.params.n_max, out=smp_p)
    assert hp.status() == (0, 0)
    hp.close()
