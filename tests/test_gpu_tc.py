"""Tensor-core (tcgen05) decode: the MMA self-test against a plain matmul,
and the decode modes against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2404_14044_b300 import scenes

pytestmark = pytest.mark.gpu


def _H():
    from paper_2404_14044_b300 import hashpoint
    return hashpoint


@pytest.mark.parametrize("K,N", [(16, 16), (32, 128), (128, 128), (64, 256), (128, 48)])
@pytest.mark.parametrize("bf16", [False, True])
@pytest.mark.parametrize("a_tmem", [False, True])
def test_mma_selftest_matches_matmul(K, N, bf16, a_tmem):
    H = _H()
    dev = torch.device("cuda", 0)
    g = torch.Generator(device="cpu").manual_seed(K * 1000 + N)
    dt = torch.bfloat16 if bf16 else torch.float16
    A = torch.randn(128, K, generator=g).to(dt)
    B = torch.randn(N, K, generator=g).to(dt)
    hp = H.HashPoint(scenes.Params(), dev)
    D = hp.selftest_mma(A.to(dev).view(torch.int16).contiguous(), B.to(dev).view(torch.int16).contiguous(), bf16,
                        a_tmem)
    assert hp.status() == (0, 0)
    ref = A.double() @ B.double().T                    # products exact in FP32; FP32 sums
    err = (D.cpu().double() - ref).abs().max().item()
    assert err <= 1e-5 * K * ref.abs().max().item() + 1e-6, err
    hp.close()


def _render(sc, decode):
    H = _H()
    dev = torch.device("cuda", 0)
    hp = H.HashPoint(sc.params, dev)
    rgb, wsum, smp = hp.render(torch.from_numpy(sc.points).to(dev), torch.from_numpy(sc.feats).to(dev), sc.camera,
                               sc.mlp_dims, torch.from_numpy(sc.mlp_params).to(dev), decode=decode)
    st = hp.status()
    R = sc.camera.width * sc.camera.height
    out = smp.packed(R)
    hp.close()
    return st, rgb.cpu().numpy().astype(np.float64), wsum.cpu().numpy().astype(np.float64), out


@pytest.mark.parametrize("which", ["sphere_plane_64", "objects_200"])
def test_decode_modes_against_oracle(which):
    H = _H()
    sc = scenes.sphere_plane_64() if which == "sphere_plane_64" else scenes.objects_800(n_points=250_000, res=200)
    o = oracle.render(sc.points, sc.feats, sc.camera, sc.params, sc.mlp_dims, sc.mlp_params, nthreads=8)
    ref = o["rgb"]
    res = {}
    for mode in (H.DECODE_FP32, H.DECODE_FP32_SIMT, H.DECODE_BF16):
        st, rgb, ws, smp = _render(sc, mode)
        assert st == (0, 0)
        assert np.array_equal(smp["n_s"].numpy(), o["n_s"])
        err = np.abs(rgb - ref)
        res[mode] = (err.max(), err.mean())
        if mode != H.DECODE_BF16:
            assert np.all(err <= 1e-4 * np.abs(ref) + 1e-6), (mode, err.max())
            assert np.all(np.abs(ws - o["wsum"]) <= 1e-4 * np.abs(o["wsum"]) + 1e-6)
        else:
            # BF16 operands (8-bit mantissa): stated error, bounded loosely
            assert err.max() < 5e-2 and err.mean() < 5e-3, res[mode]
    print(which, {k: (float(a), float(b)) for k, (a, b) in res.items()})
