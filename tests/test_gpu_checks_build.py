"""The bounds-check build (libhashpoint_checks.so, compiled with
-DHP_CHECKS=1): the hot path over the test scenes -- table build, search,
render with packed lists and with the lists left in the slots, every decode
path, the backward, the proposal's restricted search with both fallback
paths and the learned search -- records no bounds error; an out-of-range neighbour id
planted in caller-owned packed lists is reported as HP_ERR_BOUNDS with the
id, and the access is skipped.  Runs in a child process: this one has the
normal library loaded."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import sys
    import torch
    sys.path.insert(0, {root!r})
    from paper_2404_14044_b300 import build, scenes
    from paper_2404_14044_b300 import hashpoint as H
    H.LIB_PATH = build.LIB_CHECKS
    dev = torch.device("cuda", 0)

    def frame(hp, sc, lists, decode):
        R = sc.camera.width * sc.camera.height
        pts = torch.from_numpy(sc.points).to(dev)
        feats = torch.from_numpy(sc.feats).to(dev)
        mlp = torch.from_numpy(sc.mlp_params).to(dev)
        smp = H.SampleBuffers.allocate(R, sc.params.K, sc.params.n_max, dev, lists=lists)
        hp.build_table(pts, sc.camera, sc.params.r)
        hp.search_sample(None, sc.params.K, sc.params.n_max, out=smp)
        rgb, wsum = hp.aggregate_render(smp, feats, sc.mlp_dims, mlp, decode=decode)
        return pts, feats, mlp, smp, rgb

    for sc in (scenes.sphere_plane_64(), scenes.objects_800(n_points=250_000, res=200),
               scenes.forward_1008(n_field=200_000, n_occ=50_000, width=252, height=189)):
        hp = H.HashPoint(sc.params, dev)
        for lists in (True, False):
            for decode in (H.DECODE_FP32, H.DECODE_BF16, H.DECODE_FP32_SIMT):
                frame(hp, sc, lists, decode)
                assert hp.status() == (0, 0), (sc.name, lists, decode, hp.status())
        pts, feats, mlp, smp, rgb = frame(hp, sc, True, H.DECODE_FP32)
        hp.aggregate_render_backward(smp, pts, feats, sc.mlp_dims, mlp, torch.ones_like(rgb) * 1e-3)
        assert hp.status() == (0, 0), (sc.name, "backward", hp.status())
        hp.close()

    # the proposal paths: inference + restricted search + fallback (K 8: the
    # warp kernel; K 16 with every hit ray falling back: the lane kernel, then
    # the warp kernel), and the fused learned search
    for K in (8, 16):
        sc = scenes.objects_800(n_points=250_000, res=200)
        sc.params.K = K
        hp = H.HashPoint(sc.params, dev)
        pts = torch.from_numpy(sc.points).to(dev)
        feats = torch.from_numpy(sc.feats).to(dev)
        mlp = torch.from_numpy(sc.mlp_params).to(dev)
        R = sc.camera.width * sc.camera.height
        st = H.ProposalState(dev, seed=3)
        hp.build_table(pts, sc.camera, sc.params.r)
        plain = hp.search_sample(None, K, sc.params.n_max)
        packed = plain.packed(R)
        ns, off, tt = packed["n_s"], packed["sample_offset"], packed["t"]
        iv = torch.tensor([[sc.camera.t_near, sc.camera.t_far]]).repeat(R, 1)
        hit = (ns > 0).nonzero().flatten()
        iv[hit, 0] = (tt[off[hit]] + 1e-4).clamp(sc.camera.t_near, sc.camera.t_far)
        iv = iv.to(dev).contiguous()
        fb = torch.zeros(1, dtype=torch.int32, device=dev)
        smp = hp.search_sample_proposal(None, K, sc.params.n_max, iv, fallback_count=fb)
        hp.aggregate_render(smp, feats, sc.mlp_dims, mlp, decode=H.DECODE_BF16)
        assert hp.status() == (0, 0), ("restricted", K, hp.status())
        ivn = hp.proposal_infer(None, st.bf16)
        smp = hp.search_sample_proposal(None, K, sc.params.n_max, ivn, fallback_count=fb)
        smp = hp.search_sample_learned(None, K, sc.params.n_max, st.bf16)
        hp.aggregate_render(smp, feats, sc.mlp_dims, mlp)
        assert hp.status() == (0, 0), ("learned", K, hp.status())
        hp.close()

    # a neighbour id past the feature rows in the caller's packed lists
    sc = scenes.sphere_plane_64()
    hp = H.HashPoint(sc.params, dev)
    pts, feats, mlp, smp, rgb = frame(hp, sc, True, H.DECODE_FP32)
    assert hp.status() == (0, 0)
    bad = feats.shape[0] + 5
    smp.nbr[0, 0] = bad
    hp.aggregate_render(smp, feats, sc.mlp_dims, mlp, decode=H.DECODE_FP32)
    assert hp.status() == (H.HP_ERR_BOUNDS, bad), hp.status()
    hp.close()
    print("OK")
""")


def test_checks_build_clean_and_reports_a_bad_index():
    from paper_2404_14044_b300 import build
    assert os.path.exists(build.LIB_CHECKS), "build it with python -m paper_2404_14044_b300.build"
    r = subprocess.run([sys.executable, "-c", CHILD.format(root=ROOT)], capture_output=True, text=True, timeout=900)
    assert r.returncode == 0 and "OK" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]
