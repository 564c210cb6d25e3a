"""Several library contexts on several streams at once (one context per
stream, as the C-ABI asks): four views of a training step run concurrently,
each on its own stream and context, give the images of the same views run
one after another on one context bit for bit, and the same feature and
position gradients summed over the views (the backward accumulates them with
atomics, so the order of the additions, not the terms, differs)."""
import numpy as np
import pytest
import torch

from paper_2404_14044_b300 import scenes

pytestmark = pytest.mark.gpu


def test_concurrent_contexts_match_serial():
    from paper_2404_14044_b300 import hashpoint as H
    dev = torch.device("cuda", 0)
    sc = scenes.objects_800(n_points=250_000, res=200)
    p, dims = sc.params, sc.mlp_dims
    W, Hh = sc.camera.width, sc.camera.height
    cams = scenes.random_sphere_cameras(4, 4.0, 5, width=W, height=Hh)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    pts, feats, mlp = t(sc.points), t(sc.feats), t(sc.mlp_params)
    rays = [t(np.sort(scenes.random_rays(W, Hh, 2048, v)).astype(np.int32)) for v in range(4)]
    ctxs = [H.HashPoint(p, dev) for _ in range(4)]
    smps = [H.SampleBuffers.allocate(2048, p.K, p.n_max, dev) for _ in range(4)]

    def view(c, v, sm, gf, gp):
        c.build_table(pts, cams[v], p.r)
        c.search_sample(rays[v], p.K, p.n_max, out=sm)
        rgb, wsum = c.aggregate_render(sm, feats, dims, mlp)
        g = torch.full_like(rgb, 1e-3) * (v + 1)
        c.aggregate_render_backward(sm, pts, feats, dims, mlp, g, grad_feats=gf, grad_points=gp)
        return rgb

    # one context, one stream
    gf_s, gp_s = torch.zeros_like(feats), torch.zeros_like(pts)
    rgb_s = [view(ctxs[0], v, smps[0], gf_s, gp_s).clone() for v in range(4)]
    torch.cuda.synchronize()
    # four contexts on four streams
    gf_c, gp_c = torch.zeros_like(feats), torch.zeros_like(pts)
    streams = [torch.cuda.Stream() for _ in range(4)]
    main = torch.cuda.current_stream()
    fork = torch.cuda.Event()
    fork.record(main)
    rgb_c = []
    for v in range(4):
        streams[v].wait_event(fork)
        with torch.cuda.stream(streams[v]):
            rgb_c.append(view(ctxs[v], v, smps[v], gf_c, gp_c))
    for s in streams:
        main.wait_stream(s)
    torch.cuda.synchronize()
    for c in ctxs:
        assert c.status() == (0, 0)
        c.close()
    for v in range(4):
        assert torch.equal(rgb_s[v].view(torch.int32), rgb_c[v].view(torch.int32)), v
    assert float(gf_s.abs().max()) > 0 and float(gp_s.abs().max()) > 0
    assert torch.allclose(gf_c, gf_s, rtol=1e-4, atol=1e-9)
    assert torch.allclose(gp_c, gp_s, rtol=1e-4, atol=1e-9)
