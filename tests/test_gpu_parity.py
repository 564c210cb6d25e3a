"""CUDA path vs the CPU oracle, through the C-ABI.

Bit-exact on every discrete output (table, neighbour sets, sample depths and
sources, primary bucket keys, sample counts); colours within
|d| <= 1e-4 |ref| + 1e-6 per channel (FP32 path vs the FP64 oracle)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2404_14044_b300 import scenes

pytestmark = pytest.mark.gpu

RTOL, ATOL = 1e-4, 1e-6


def _H():
    from paper_2404_14044_b300 import hashpoint
    return hashpoint


def gpu_render(sc, rays=None, params=None, capacity=None, points=None, feats=None):
    H = _H()
    p = params or sc.params
    dev = torch.device("cuda", 0)
    pts = torch.from_numpy(points if points is not None else sc.points).to(dev)
    fts = torch.from_numpy(feats if feats is not None else sc.feats).to(dev)
    mlp = torch.from_numpy(sc.mlp_params).to(dev)
    hp = H.HashPoint(p, dev)
    R = sc.camera.width * sc.camera.height if rays is None else len(rays)
    hp.reserve(sc.camera, p.r, len(pts), R, p.n_max)
    rt = None if rays is None else torch.from_numpy(np.ascontiguousarray(rays, np.int32)).to(dev)
    smp = None
    if capacity is not None:
        smp = H.SampleBuffers.allocate(R, p.K, p.n_max, dev, capacity=capacity)
    rgb, wsum, smp = hp.render(pts, fts, sc.camera, sc.mlp_dims, mlp, rays=rt, samples=smp)
    status = hp.status()
    out = smp.packed(R)
    out["rgb"] = rgb.cpu().numpy().astype(np.float64)
    out["wsum"] = wsum.cpu().numpy().astype(np.float64)
    out["status"] = status
    tb = hp.table()
    out["table"] = dict(h=tb["h"], start=tb["start"].cpu().numpy().view(np.uint32), points=tb["points"].cpu().numpy())
    hp.close()
    return {k: (v.numpy() if isinstance(v, torch.Tensor) else v) for k, v in out.items()}


def oracle_render(sc, rays=None, params=None, points=None, feats=None):
    p = params or sc.params
    return oracle.render(sc.points if points is None else points, sc.feats if feats is None else feats, sc.camera,
                         p, sc.mlp_dims, sc.mlp_params, rays=rays, nthreads=8)


def assert_parity(g, o, K, check_table=None):
    assert g["status"] == (0, 0), g["status"]
    assert g["S"] == o["S"]
    for k in ("n_s", "primary", "cand_count", "sample_offset", "t", "src", "nbr", "nbr_dist"):
        a, b = np.asarray(g[k]), np.asarray(o[k])
        assert a.shape == b.shape, (k, a.shape, b.shape)
        if a.dtype.kind == "f":
            assert np.array_equal(a.view(np.int32), b.astype(np.float32).view(np.int32)), k
        else:
            assert np.array_equal(a, b), (k, np.nonzero(a != b)[0][:10])
    assert np.array_equal(g["ray"], o["ray"])
    # interval to the next sample (exact float32 difference), 2 r(t) for the last
    off = o["sample_offset"]
    for i in np.nonzero(o["n_s"] > 1)[0][:500]:
        a, b = off[i], off[i + 1]
        assert np.array_equal(g["delta"][a:b - 1], (o["t"][a + 1:b] - o["t"][a:b - 1]).astype(np.float32))
    err = np.abs(g["rgb"] - o["rgb"])
    lim = RTOL * np.abs(o["rgb"]) + ATOL
    assert np.all(err <= lim), (err.max(), np.argmax(err - lim))
    assert np.all(np.abs(g["wsum"] - o["wsum"]) <= RTOL * np.abs(o["wsum"]) + ATOL)
    assert np.all(g["wsum"] <= 1.0 + 1e-6) and np.all(g["wsum"] >= 0.0)


def assert_table(g, sc, params=None, points=None):
    tb = oracle.build_table(sc.points if points is None else points, sc.camera, params or sc.params)
    gt = g["table"]
    assert gt["h"] == tb["h"]
    assert np.array_equal(gt["start"], tb["start"])
    nv = tb["n_visible"]
    gp = gt["points"][:nv]
    assert np.array_equal(gp[:, :3].view(np.int32), tb["pos"].view(np.int32))
    assert np.array_equal(gp[:, 3].view(np.int32), tb["ids"])


# ------------------------------------------------------------- full frames

def test_sphere_plane_64_full_frame():
    sc = scenes.sphere_plane_64()
    g = gpu_render(sc)
    o = oracle_render(sc)
    assert_parity(g, o, sc.params.K)
    assert_table(g, sc)
    assert o["S"] > 4000 and (o["n_s"] == 0).sum() > 100        # hits and misses both present


def _tiny(mode, res=48, n=20000, seed=0, **kw):
    sc = scenes.sphere_plane_64(seed=seed, n_sphere=n // 2, n_plane=n // 2, res=res)
    p = scenes.Params(**{**sc.params.__dict__, "radius_mode": mode, "rho": 2.5 if mode else 0.0, **kw})
    sc.params = p
    return sc


@pytest.mark.parametrize("mode", [scenes.RADIUS_FIXED, scenes.RADIUS_CONE_EXACT, scenes.RADIUS_CONE_APPROX])
def test_radius_modes(mode):
    sc = _tiny(mode)
    g = gpu_render(sc)
    o = oracle_render(sc)
    assert_parity(g, o, sc.params.K)
    assert_table(g, sc)


@pytest.mark.parametrize("kw", [dict(K=1, n_max=1), dict(K=16, n_max=8, gamma=0.5), dict(K=32, n_max=16, gamma=0.2),
                                dict(bg_mode=1), dict(cand_cap=3), dict(gap_k=1.0, gamma=0.3), dict(eps_w=0.0, n_max=16)])
def test_parameter_variants(kw):
    sc = _tiny(scenes.RADIUS_FIXED, res=40, n=16000, seed=2, **kw)
    g = gpu_render(sc)
    o = oracle_render(sc)
    assert_parity(g, o, sc.params.K)


def test_gamma_transition_parity():
    # gap_k = 0: no cluster gate; lowering gamma moves sampling from the primary
    # surface onto the surfaces behind it (multi-surface), bit-exact at every gamma
    sc = scenes.objects_800(n_points=1_000_000, res=160)
    base = sc.params
    S = []
    for gamma in (0.9, 0.5, 0.2, 0.05):
        sc.params = scenes.Params(**{**base.__dict__, "gamma": gamma, "gap_k": 0.0, "n_max": 16})
        g = gpu_render(sc)
        o = oracle_render(sc)
        assert_parity(g, o, sc.params.K)
        S.append(o["S"])
    assert S == sorted(S) and S[-1] > 2 * S[0]


def test_mlp_shapes():
    sc = _tiny(scenes.RADIUS_FIXED, res=32, n=8000)
    for dims in ([32, 4], [32, 16, 4], [32, 128, 128, 128, 4], [32, 32, 64, 16, 128, 4]):
        sc.mlp_dims = dims
        sc.mlp_params = scenes.random_mlp(dims, 5, sigma_bias=60.0)
        g = gpu_render(sc)
        o = oracle_render(sc)
        assert_parity(g, o, sc.params.K)


@pytest.mark.parametrize("K", [8, 16])
def test_wide_mlp_neighbour_counts(K):
    # the widest supported MLP with 8 and 16 neighbours: the neighbour lists
    # and the split weights together nearly fill the decode's shared memory
    sc = _tiny(scenes.RADIUS_FIXED, res=32, n=8000, K=K, n_max=8)
    sc.mlp_dims = [32, 128, 128, 128, 4]
    sc.mlp_params = scenes.random_mlp(sc.mlp_dims, 6, sigma_bias=60.0)
    g = gpu_render(sc)
    o = oracle_render(sc)
    assert_parity(g, o, sc.params.K)


def test_feature_widths():
    sc = _tiny(scenes.RADIUS_FIXED, res=32, n=8000)
    for F in (4, 16, 64, 128):
        feats = scenes.random_features(len(sc.points), F, 3)
        sc.feats = feats
        sc.mlp_dims = [F, 32, 4]
        sc.mlp_params = scenes.random_mlp(sc.mlp_dims, 1, sigma_bias=60.0)
        g = gpu_render(sc)
        o = oracle_render(sc)
        assert_parity(g, o, sc.params.K)


def test_ray_subset_ragged_and_repeated():
    sc = scenes.sphere_plane_64()
    rng = np.random.default_rng(3)
    rays = rng.integers(0, 64 * 64, 1000).astype(np.int32)        # ragged count, repeats allowed
    g = gpu_render(sc, rays=rays)
    o = oracle_render(sc, rays=rays)
    assert_parity(g, o, sc.params.K)


def test_objects_reduced_full_frame():
    # the at-scale scene shrunk so the oracle renders every ray in seconds
    sc = scenes.objects_800(n_points=250_000, res=200)
    g = gpu_render(sc)
    o = oracle_render(sc)
    assert_parity(g, o, sc.params.K)
    assert_table(g, sc)


@pytest.mark.parametrize("mode,K,n", [(scenes.RADIUS_FIXED, 8, 250_000), (scenes.RADIUS_FIXED, 16, 250_000),
                                      (scenes.RADIUS_CONE_EXACT, 16, 120_000), (scenes.RADIUS_FIXED, 32, 250_000),
                                      (scenes.RADIUS_FIXED, 3, 250_000)])
def test_crowded_rays_full_frame(mode, K, n):
    # dense clouds: rays with more candidates than a lane's column (48) and
    # than the point-major pass's slots (128), so the warp-per-ray search runs
    # both from the slots and with its own walk
    sc = scenes.sphere_plane_64(seed=3, n_sphere=n // 2, n_plane=n // 2, res=64)
    sc.params = scenes.Params(**{**sc.params.__dict__, "radius_mode": mode, "rho": 2.5 if mode else 0.0, "K": K})
    g = gpu_render(sc)
    o = oracle_render(sc)
    c = np.asarray(o["cand_count"])
    assert (c > 48).sum() > 500 and (c > 128).sum() > 100 and ((c > 48) & (c <= 128)).sum() > 500
    assert_parity(g, o, sc.params.K)
    assert_table(g, sc)


# ------------------------------------------- full-size workloads, sampled rays

def _sampled(sc, n=3000, seed=11):
    g = gpu_render(sc)                                   # every ray, the benchmark's launch configuration
    rays = np.sort(np.random.default_rng(seed).choice(sc.camera.width * sc.camera.height, n, replace=False))
    o = oracle_render(sc, rays=rays.astype(np.int32))
    gs = {}
    off = g["sample_offset"]
    sel = np.concatenate([np.arange(off[i], off[i + 1]) for i in rays]).astype(np.int64)
    for k in ("n_s", "primary", "cand_count"):
        gs[k] = g[k][rays]
    gs["sample_offset"] = np.concatenate([[0], np.cumsum(gs["n_s"])]).astype(np.int64)
    for k in ("t", "src", "nbr", "nbr_dist", "delta"):
        gs[k] = g[k][sel]
    gs["ray"] = np.repeat(np.arange(len(rays)), gs["n_s"]).astype(np.int32)
    gs["S"] = int(gs["sample_offset"][-1])
    gs["rgb"], gs["wsum"], gs["status"] = g["rgb"][rays], g["wsum"][rays], g["status"]
    assert_parity(gs, o, sc.params.K)
    return g, o


def test_objects_800_full_size_sampled():
    sc = scenes.objects_800()
    g, o = _sampled(sc)
    assert o["S"] > 1000
    # whole-frame properties at full size
    assert np.array_equal(np.diff(g["sample_offset"]), g["n_s"])
    assert np.all((g["n_s"] == 0) == (g["cand_count"] == 0))
    assert g["table"]["start"][-1] <= len(sc.points)


def test_forward_1008_full_size_sampled():
    sc = scenes.forward_1008()
    g, o = _sampled(sc, n=2000)
    assert o["S"] > 1000


# ----------------------------------------------------------------- edge cases

def test_no_points_and_no_rays():
    sc = scenes.sphere_plane_64()
    empty = np.zeros((0, 3), np.float32)
    g = gpu_render(sc, points=empty, feats=np.zeros((0, 32), np.float32))
    assert g["S"] == 0 and np.all(g["n_s"] == 0) and np.all(g["primary"] == -1) and np.all(g["rgb"] == 0)
    assert g["status"] == (0, 0)
    g = gpu_render(sc, rays=np.zeros(0, np.int32))
    assert g["S"] == 0 and g["status"] == (0, 0)


def test_single_point():
    sc = scenes.sphere_plane_64()
    # on the ray through the centre of pixel (32, 32), 3 units from the camera
    d = np.array([0.5 / sc.camera.fx, 0.5 / sc.camera.fy, 1.0])
    d /= np.linalg.norm(d)
    pt = (sc.camera.eye() + 3.0 * (np.asarray(sc.camera.R, np.float64).T @ d)).astype(np.float32)[None]
    g = gpu_render(sc, points=pt, feats=sc.feats[:1])
    o = oracle_render(sc, points=pt, feats=sc.feats[:1])
    assert_parity(g, o, sc.params.K)
    assert o["S"] >= 1


def test_bad_ray_reported_not_faulted():
    sc = scenes.sphere_plane_64()
    rays = np.array([5, 64 * 64, -1, 7], np.int32)
    g = gpu_render(sc, rays=rays)
    assert g["status"][0] == _H().HP_ERR_BAD_RAY
    assert g["n_s"][1] == 0 and g["n_s"][2] == 0


def test_sample_capacity_overflow_reported():
    sc = scenes.sphere_plane_64()
    g = gpu_render(sc, capacity=100)
    assert g["status"][0] == _H().HP_ERR_OVERFLOW
    o = oracle_render(sc)
    n = 100
    assert np.array_equal(g["t"][:n], o["t"][:n].astype(np.float32))


def test_deterministic_and_permutation_invariant():
    sc = _tiny(scenes.RADIUS_FIXED, res=64, n=30000, seed=4)
    a = gpu_render(sc)
    b = gpu_render(sc)
    for k in ("n_s", "primary", "t", "src", "nbr", "nbr_dist", "rgb"):
        assert np.array_equal(a[k], b[k]), k
    perm = np.random.default_rng(0).permutation(len(sc.points))
    c = gpu_render(sc, points=sc.points[perm], feats=sc.feats[perm])
    assert np.array_equal(a["n_s"], c["n_s"]) and np.array_equal(a["t"], c["t"])
    assert np.array_equal(a["src"], perm[c["src"]])
    assert np.array_equal(a["rgb"], c["rgb"])
    assert np.array_equal(a["table"]["start"], c["table"]["start"])


def test_bounded_wait_gives_up_without_hanging():
    # the scan tile 0 never publishes; its successor gives up after a short spin
    H = _H()
    sc = scenes.objects_800(n_points=50_000, res=200)
    dev = torch.device("cuda", 0)
    hp = H.HashPoint(sc.params, dev)
    pts = torch.from_numpy(sc.points).to(dev)
    hp.debug_fault(0, 2000)
    hp.build_table(pts, sc.camera, sc.params.r)
    code, detail = hp.status()
    assert code == H.HP_ERR_TIMEOUT and detail >= 1                   # a tile after the silent one
    hp.debug_fault(-1, 0)                                           # context still usable
    hp.build_table(pts, sc.camera, sc.params.r)
    assert hp.status() == (0, 0)
    hp.close()
