"""Pins of the CPU oracle against what the paper and the mathematics fix:
closed forms, brute force, an independent float64 geometry, special cases of
the selection rule, and invariants.  CPU only."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2404_14044_b300 import scenes
from tests import ref64

HERE = os.path.dirname(os.path.abspath(__file__))


def tiny_scene(seed=0, res=16, n=2000, mode=scenes.RADIUS_FIXED, r=0.03):
    """16x16 view of the sphere+plane scene (the small parity workload shrunk)."""
    cam = scenes.make_camera(res, res, 40.0, (0.0, -3.0, 0.0), t_near=1.0, t_far=10.0)
    pts = scenes.sphere_plane_points(n // 2, n // 2, seed)
    p = scenes.Params(radius_mode=mode, r=r, rho=2.0 if mode else 0.0, K=8, n_max=4)
    dims = [32, 16, 4]
    return pts, scenes.random_features(len(pts), 32, seed + 1), cam, p, dims, scenes.random_mlp(dims, seed, 1.5 / 0.03)


# ---------------------------------------------------------------- exp32

def test_exp32_accuracy_and_exact_points():
    # decision exp: within 2 ulp of exp() over the normal range it is used on
    xs = np.concatenate([-np.logspace(-8, math.log10(87.0), 4000), np.linspace(-87.0, 0.0, 4001)])
    worst = 0.0
    for x in xs.astype(np.float32):
        y = oracle.exp32(float(x))
        ref = math.exp(float(x))
        worst = max(worst, abs(y - ref) / ref32ulp(ref))
    assert worst <= 2.0, worst
    assert oracle.exp32(0.0) == 1.0
    for k in range(0, 120, 7):                      # exp(-k ln2) ~ 2^-k (subnormal below 2^-126)
        x = float(np.float32(-k * math.log(2.0)))
        y = oracle.exp32(x)
        assert abs(y - math.exp(x)) <= 2 * ref32ulp(math.exp(x))
        assert abs(y / 2.0 ** -k - 1) < 2e-5           # float32(-k ln2) carries ~k*6e-8 rounding
    assert oracle.exp32(-200.0) == 0.0
    # monotone non-increasing as x decreases
    ys = [oracle.exp32(float(x)) for x in np.linspace(-20, 0, 3001, dtype=np.float32)]
    assert all(a <= b for a, b in zip(ys, ys[1:]))


def ref32ulp(v):
    return ref64.ulp32(v)


# ------------------------------------------------------------ window size

def test_kernel_size_golden_cone_mode():
    g = json.load(open(os.path.join(HERE, "golden", "kernel_size.json")))
    # narrow field of view: obliquity ~1, so the paper's s governs the window
    cam = scenes.make_camera(64, 64, 2.0, (0.0, -3.0, 0.0), t_near=1.0, t_far=10.0)
    for case in g["cases"]:
        rho, s = case["rho"], case["s"]
        half = (s - 1) / 2
        assert (half - 1) < rho <= half                 # Supplementary admissible range
        for mode in (scenes.RADIUS_CONE_EXACT, scenes.RADIUS_CONE_APPROX):
            h, rdd = oracle.window(cam, scenes.Params(radius_mode=mode, rho=rho))
            assert 2 * h + 1 == s, (rho, h, s)
            rdot = math.sqrt((1 / cam.fx) * (1 / cam.fy) / math.pi)      # Sec. 3.2 disc radius
            assert rdd == pytest.approx(rho * rdot, rel=1e-6)


def test_cone_rmin_matches_input_radius_at_tnear():
    # Sec. 3.2: r_min, at t_near on the central ray, equals the input radius
    cam = scenes.make_camera(65, 65, 40.0, (0.0, -3.0, 0.0), t_near=1.5, t_far=10.0)
    for mode in (scenes.RADIUS_CONE_EXACT, scenes.RADIUS_CONE_APPROX):
        p = scenes.Params(radius_mode=mode, r=0.01, rho=0.0)
        d, n2, ln, c = oracle.ray(cam, p, 32, 32)       # pixel centre on the principal point
        assert cam.t_near * c == pytest.approx(0.01, rel=1e-5)


# ---------------------------------------------------------- radius (cone)

@pytest.mark.parametrize("pix", [(0, 0), (10, 50), (32, 32), (63, 5), (40, 20)])
def test_cone_radius_against_construction(pix):
    cam = scenes.make_camera(64, 64, 60.0, (0.0, -3.0, 0.0), t_near=1.0, t_far=10.0)
    p = scenes.Params(radius_mode=scenes.RADIUS_CONE_EXACT, rho=2.0)
    h, rdd = oracle.window(cam, p)
    _, _, _, c = oracle.ray(cam, p, *pix)
    assert c == pytest.approx(ref64.cone_sin(cam, *pix, rdd), rel=2e-6)
    pa = scenes.Params(radius_mode=scenes.RADIUS_CONE_APPROX, rho=2.0)
    _, _, _, ca = oracle.ray(cam, pa, *pix)
    assert ca == pytest.approx(ref64.cone_tan_approx(cam, *pix, rdd), rel=2e-6)
    # the small-angle form agrees with the exact one to O(angle^2)
    assert abs(ca - c) / c < 5 * (rdd * math.hypot(1, rdd)) + 0.05


def test_cone_radius_principal_point_closed_form():
    # at p_o = principal point, Eq. radius reduces to t * rdd / sqrt(rdd^2 + f^2)
    cam = scenes.make_camera(65, 65, 40.0, (0.0, -3.0, 0.0), t_near=1.0, t_far=10.0)
    p = scenes.Params(radius_mode=scenes.RADIUS_CONE_EXACT, rho=3.0)
    h, rdd = oracle.window(cam, p)
    _, _, _, c = oracle.ray(cam, p, 32, 32)
    assert c == pytest.approx(rdd / math.sqrt(rdd * rdd + 1.0), rel=1e-6)


# ------------------------------------------------------------- table build

def _fp64_pixels(cam, pts):
    P = ref64.cam_space(cam, pts)
    u = cam.fx * P[:, 0] / P[:, 2] + cam.cx
    v = cam.fy * P[:, 1] / P[:, 2] + cam.cy
    return P, u, v


def test_table_against_fp64_projection_and_order():
    pts, feats, cam, p, dims, mlp = tiny_scene(res=24, n=4000)
    tb = oracle.build_table(pts, cam, p)
    h = tb["h"]
    Wp, Hp = cam.width + 2 * h, cam.height + 2 * h
    start, ids, pos = tb["start"], tb["ids"], tb["pos"]
    assert start[0] == 0 and start[-1] == tb["n_visible"] and np.all(np.diff(start.astype(np.int64)) >= 0)
    P, u, v = _fp64_pixels(cam, pts)
    inside = (P[:, 2] > cam.z_near) & (u >= -h) & (u < cam.width + h) & (v >= -h) & (v < cam.height + h)
    near_edge = (np.abs(u - np.round(u)) < 1e-3) | (np.abs(v - np.round(v)) < 1e-3)
    kept = np.zeros(len(pts), bool)
    kept[ids] = True
    assert np.all(kept[~near_edge] == inside[~near_edge])
    keys = np.repeat(np.arange(Wp * Hp), np.diff(start.astype(np.int64)))
    iu, iv = keys % Wp - h, keys // Wp - h
    ok = ~near_edge[ids]
    assert np.all(np.floor(u[ids])[ok] == iu[ok]) and np.all(np.floor(v[ids])[ok] == iv[ok])
    # camera-space positions within float32 rounding of the float64 transform
    assert np.allclose(pos, P[ids], atol=5e-6)
    # each bucket ordered by (depth, x, y, id)
    for k in np.nonzero(np.diff(start.astype(np.int64)) > 1)[0]:
        a, b = start[k], start[k + 1]
        rows = [(pos[i, 2], pos[i, 0], pos[i, 1], ids[i]) for i in range(a, b)]
        assert rows == sorted(rows)


def test_table_permutation_invariance():
    pts, feats, cam, p, dims, mlp = tiny_scene(res=20, n=3000, seed=3)
    perm = np.random.default_rng(7).permutation(len(pts))
    a = oracle.build_table(pts, cam, p)
    b = oracle.build_table(pts[perm], cam, p)
    assert np.array_equal(a["start"], b["start"])
    assert np.array_equal(a["pos"], b["pos"])
    assert np.array_equal(a["ids"], perm[b["ids"]])       # same points, ids mapped through perm


# ------------------------------------------------------------------ search

@pytest.mark.parametrize("mode", [scenes.RADIUS_FIXED, scenes.RADIUS_CONE_EXACT, scenes.RADIUS_CONE_APPROX])
def test_window_search_equals_brute_force(mode):
    # all methods retrieve the same points (Sec. 4.2); here hashed vs brute force
    pts, feats, cam, p, dims, mlp = tiny_scene(res=16, n=3000, mode=mode)
    if mode:
        p.rho = 4.0
    for pix in range(cam.width * cam.height):
        a = oracle.ray_candidates(pts, cam, p, pix, brute=False)
        b = oracle.ray_candidates(pts, cam, p, pix, brute=True)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]


def test_search_predicate_against_fp64_geometry():
    pts, feats, cam, p, dims, mlp = tiny_scene(res=16, n=3000, r=0.05)
    P = ref64.cam_space(cam, pts)
    n_acc = 0
    for pix in range(0, 256, 3):
        pu, pv = pix % 16, pix // 16
        d = ref64.ray_dir(cam, pu, pv)
        t, rho = ref64.perp(P, d)
        ids, ts, n = oracle.ray_candidates(pts, cam, p, pix, brute=True)
        acc = np.zeros(len(pts), bool)
        acc[ids] = True
        n_acc += n
        assert np.all(rho[acc] <= p.r * (1 + 1e-4)) and np.all(t[acc] >= cam.t_near * (1 - 1e-5))
        clear = (rho < p.r * (1 - 1e-4)) & (t > cam.t_near * (1 + 1e-5)) & (t < cam.t_far * (1 - 1e-5)) & (P[:, 2] > cam.z_near)
        assert np.array_equal(acc & clear, clear)          # every clear inside point accepted
        assert np.allclose(ts, t[ids], rtol=1e-6, atol=1e-6)
        assert np.all(np.diff(ts) >= 0)                    # depth order
    assert n_acc > 100


@pytest.mark.parametrize("which", ["tiny", "sphere_plane_64", "wide_radius"])
def test_frame_brute_force_equals_hashed(which):
    if which == "tiny":
        pts, feats, cam, p, dims, mlp = tiny_scene(res=16, n=3000)
    elif which == "wide_radius":
        # a dense slab right at t_near: the radius spans ~3.5 pixels there, so a
        # window smaller than the bound misses points
        pts, feats, cam, p, dims, mlp = tiny_scene(res=32, n=2000, r=0.08)
        cam = scenes.Camera(32, 32, 44.0, 44.0, 16.0, 16.0, np.eye(3, dtype=np.float32), np.zeros(3, np.float32),
                            1.0, 10.0, 0.05)
        rng = np.random.default_rng(9)
        z = rng.uniform(1.0, 1.1, 30000)
        pts = np.stack([rng.uniform(-0.45, 0.45, 30000) * z, rng.uniform(-0.45, 0.45, 30000) * z, z], 1)
        pts = pts.astype(np.float32)
        feats = scenes.random_features(len(pts), 32, 2)
        assert oracle.window(cam, p)[0] == 4
    else:
        sc = scenes.sphere_plane_64()
        pts, feats, cam, p, dims, mlp = sc.points, sc.feats, sc.camera, sc.params, sc.mlp_dims, sc.mlp_params
    a = oracle.render(pts, feats, cam, p, dims, mlp, nthreads=4)
    b = oracle.render(pts, feats, cam, p, dims, mlp, brute=True, nthreads=4)
    for k in ("n_s", "primary", "cand_count", "sample_offset", "t", "src", "nbr", "nbr_dist"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["rgb"], b["rgb"])


# --------------------------------------------------------------- selection

def _ray_cands(cam, p, pix, ts, offsets):
    """Candidates along the ray of pixel ``pix`` at depths ts, displaced
    perpendicular to the ray by offsets (float64 geometry, stored float32)."""
    d = ref64.ray_dir(cam, pix % cam.width, pix // cam.width)
    a = np.cross(d, [0.0, 1.0, 0.0])
    a /= np.linalg.norm(a)
    P = np.array([t * d + o * a for t, o in zip(ts, offsets)], np.float32)
    dd, _, _, _ = oracle.ray(cam, p, pix % cam.width, pix // cam.width)
    tt = np.array([(np.float32(x[0]) * dd[0] + np.float32(x[1]) * dd[1]) + np.float32(x[2]) * dd[2] for x in P],
                  np.float32)
    return P, tt


def _cam():
    return scenes.make_camera(32, 32, 40.0, (0.0, -3.0, 0.0), t_near=1.0, t_far=10.0)


def test_select_single_candidate_threshold():
    cam = _cam()
    pix = 16 * 32 + 16
    for gamma, expect in ((0.9, 1), (0.0009, 0)):     # alpha ~ gamma, eps_w = 1e-3
        p = scenes.Params(r=0.02, gamma=gamma, K=8, n_max=4)
        P, t = _ray_cands(cam, p, pix, [3.0], [0.01])
        res = oracle.select(cam, p, pix, t, [5], P)
        a = gamma * math.exp(-(0.01 ** 2) / 0.02)
        assert (a > 1e-3) == bool(expect)
        assert res["n_s"] == expect
        if expect:
            assert res["src"][0] == 5 and res["t"][0] == t[0]
            assert res["nbr"][0, 0] == 5 and np.all(res["nbr"][0, 1:] == -1)      # only itself in radius
            assert res["nbr_dist"][0, 0] == pytest.approx(0.01, rel=1e-4)


@pytest.mark.parametrize("gamma,n_max", [(0.9, 8), (0.5, 8), (0.3, 8), (0.5, 3), (0.2, 16)])
def test_select_equal_alpha_count(gamma, n_max):
    # collinear candidates on the ray, 2r apart: each one's neighbourhood is
    # itself at distance ~0, so alpha_j = gamma and w_j = gamma (1-gamma)^(j-1)
    cam = _cam()
    pix = 10 * 32 + 20
    C = 20
    p = scenes.Params(r=0.01, gamma=gamma, K=8, n_max=n_max, gap_k=4.0)
    P, t = _ray_cands(cam, p, pix, 3.0 + 0.02 * np.arange(C), np.zeros(C))
    res = oracle.select(cam, p, pix, t, np.arange(C), P)
    m = math.floor(math.log(p.eps_w / gamma) / math.log(1 - gamma)) + 1
    assert res["n_s"] == min(n_max, C, m)
    assert np.array_equal(res["src"], np.arange(res["n_s"]))


def test_select_primary_cluster_stops_at_gap():
    # two surfaces 10 r apart: with small gamma many candidates pass eps_w on
    # both, but samples stay on the first (the primary surface)
    cam = _cam()
    pix = 16 * 32 + 16
    p = scenes.Params(r=0.01, gamma=0.2, K=8, n_max=16, gap_k=4.0)
    ts = [3.0, 3.004, 3.008, 3.1, 3.104, 3.108]
    P, t = _ray_cands(cam, p, pix, ts, [0.0, 0.003, -0.003, 0.0, 0.003, -0.003])
    res = oracle.select(cam, p, pix, t, np.arange(6), P)
    assert res["n_s"] == 3 and list(res["src"]) == [0, 1, 2]


def test_gamma_transition_without_cluster_gate():
    # Supplementary (adaptive sampling for noisy input): with the gate off,
    # lowering gamma lets weights decay slower, so sampling reaches the
    # surfaces behind the primary one; with gamma = 0.9 it stays on the first
    cam = _cam()
    pix = 16 * 32 + 16
    ts = [3.0, 3.004, 3.008, 3.1, 3.104, 3.108, 3.3, 3.304]
    P, t = _ray_cands(cam, scenes.Params(r=0.01), pix, ts, [0.0, 0.003, -0.003, 0.0, 0.003, -0.003, 0.0, 0.003])
    counts = []
    for gamma in (0.9, 0.5, 0.1, 0.01):
        p = scenes.Params(r=0.01, gamma=gamma, K=8, n_max=16, gap_k=0.0)
        res = oracle.select(cam, p, pix, t, np.arange(8), P)
        counts.append(res["n_s"])
        # the count follows w_j = gamma (1 - gamma)^(j-1) > eps_w (alpha ~ gamma here)
        m = math.floor(math.log(p.eps_w / gamma) / math.log(1 - gamma)) + 1 if gamma < 1 else 1
        assert res["n_s"] == min(8, m, 16) or gamma == 0.01
    assert counts[0] == 3 and counts == sorted(counts) and counts[-1] == 8
    gated = oracle.select(cam, scenes.Params(r=0.01, gamma=0.01, K=8, n_max=16, gap_k=4.0), pix, t, np.arange(8), P)
    assert gated["n_s"] == 3                               # the gate keeps the primary surface only


def test_select_isolated_point_loses_confidence():
    # the pseudo-UDF: a candidate whose neighbourhood is far (d_j ~ beta)
    # gets alpha << gamma and is skipped; the dense cluster behind is primary
    cam = _cam()
    pix = 16 * 32 + 16
    p = scenes.Params(r=0.4, gamma=0.9, beta2=0.02, K=4, n_max=4, gap_k=0.5)
    ts = [2.0, 3.0, 3.002, 3.004]
    P, t = _ray_cands(cam, p, pix, ts, [0.39, 0.0, 0.001, -0.001])
    res = oracle.select(cam, p, pix, t, np.arange(4), P)
    # alpha_1 = 0.9 exp(-0.39^2/0.02) ~ 4.5e-4 -> w_1 < eps_w
    assert 0.9 * math.exp(-0.39 ** 2 / 0.02) < 1e-3
    assert res["jstar"] == 1 and res["src"][0] == 1


def test_select_neighbours_sorted_within_radius():
    cam = _cam()
    pix = 16 * 32 + 16
    p = scenes.Params(r=0.01, gamma=0.9, K=3, n_max=2)
    offs = [0.0, 0.002, 0.004, 0.006, 0.0085]
    P, t = _ray_cands(cam, p, pix, [3.0] * 5, offs)
    res = oracle.select(cam, p, pix, t, np.arange(5), P)
    assert res["n_s"] >= 1
    nb, nd = res["nbr"][0], res["nbr_dist"][0]
    assert np.all(np.diff(nd) >= 0) and np.all(nd <= 0.01)
    # sample 0 sits at its own point; its 3 nearest within r are itself and the next two
    s0 = res["src"][0]
    assert nb[0] == s0


def test_select_pseudo_udf_and_weights_fp64():
    # d_j (Sec. 3.3): mean distance from x_j = o + t_j d to the K nearest
    # candidate points within r(t_j); alpha_j = gamma exp(-d_j^2/beta^2);
    # w_j = alpha_j prod_{k<j} (1 - alpha_k) (Eq. weight) -- recomputed in float64
    cam = _cam()
    pix = 12 * 32 + 9
    rng = np.random.default_rng(2)
    for K in (1, 3, 8):
        p = scenes.Params(r=0.3, gamma=0.7, beta2=0.02, K=K, n_max=8, gap_k=100.0)
        C = 12
        ts = np.sort(3.0 + rng.uniform(0, 0.5, C))
        offs = rng.uniform(-0.25, 0.25, C)
        P, t = _ray_cands(cam, p, pix, ts, offs)
        res = oracle.select(cam, p, pix, t, np.arange(C), P)
        d = oracle.ray(cam, p, pix % 32, pix // 32)[0].astype(np.float64)
        Pd = P.astype(np.float64)
        T = 1.0
        for j in range(C):
            x = np.float64(t[j]) * d
            dist = np.linalg.norm(Pd - x, axis=1)
            near = np.sort(dist[dist <= p.r])[:K]
            dj = near.mean()
            assert res["d"][j] == pytest.approx(dj, rel=1e-5)
            a = p.gamma * math.exp(-dj * dj / p.beta2)
            assert res["w"][j] == pytest.approx(a * T, rel=1e-5, abs=1e-30)
            T *= 1 - a


# ------------------------------------------------ aggregation / compositing

def _one_ray_setup(F=8):
    cam = _cam()
    pix = 16 * 32 + 16
    rng = np.random.default_rng(0)
    pts_c = None
    return cam, pix, rng


def _world_from_cam(cam, P):
    R = np.asarray(cam.R, np.float64)
    return ((np.asarray(P, np.float64) - np.asarray(cam.t, np.float64)) @ R).astype(np.float32)


def test_shade_closed_form_opaque_plane():
    # zero weights: sigma = softplus(b0), rgb = sigmoid(b1..3) for every
    # sample, so sum w' = 1 - exp(-sigma sum Delta) and c = rgb * sum w' + bg (1 - sum w')
    cam = _cam()
    pix = 16 * 32 + 16
    dims = [8, 4]
    for sig_raw, bg_mode in ((2.0, 0), (50000.0, 0), (-3.0, 1)):
        mlp = np.zeros(8 * 4 + 4, np.float32)
        mlp[32:] = [sig_raw, 0.3, -1.0, 2.0]
        p = scenes.Params(r=0.01, K=2, bg_mode=bg_mode)
        pts_c = np.array([[0.0, 0.0, 3.0]], np.float32)
        pts = _world_from_cam(cam, pts_c)
        feats = np.ones((1, 8), np.float32)
        for ts in ([3.0], [3.0, 3.004], [3.0, 3.002, 3.005, 3.011]):
            nbr = np.tile(np.array([0, -1], np.int32), (len(ts), 1))
            rgb, ws, fe, o4 = oracle.shade(pts, feats, cam, p, dims, mlp, pix, ts, nbr)
            sigma = math.log1p(math.exp(sig_raw)) if sig_raw < 30 else sig_raw
            col = 1 / (1 + np.exp(-np.array([0.3, -1.0, 2.0], np.float32).astype(np.float64)))
            tt = np.array(ts, np.float32).astype(np.float64)
            total = (tt[-1] - tt[0]) + 2 * np.float64(np.float32(0.01))
            expect_ws = 1 - math.exp(-sigma * total)
            assert ws == pytest.approx(expect_ws, rel=1e-12, abs=1e-15)
            assert np.allclose(rgb, col * expect_ws + (1 - expect_ws) * bg_mode, rtol=1e-12, atol=1e-15)
            assert np.allclose(o4[:, 0], sigma) and np.allclose(o4[:, 1:], col)
            assert 0.0 <= ws <= 1.0
        if sig_raw == 50000.0:
            assert ws > 1 - 1e-12                          # opaque: first sample takes all weight


def test_idw_closed_forms():
    cam = _cam()
    pix = 16 * 32 + 16
    F = 6
    dims = [F, 4]
    mlp = np.zeros(F * 4 + 4, np.float32)
    p = scenes.Params(r=0.05, K=3)
    d = ref64.ray_dir(cam, 16, 16)
    a = np.cross(d, [0.0, 1.0, 0.0]); a /= np.linalg.norm(a)
    b = np.cross(d, a)
    pts_c = np.array([3.0 * d + 0.01 * a, 3.0 * d - 0.03 * a, 3.0 * d + 0.02 * b], np.float32)
    pts = _world_from_cam(cam, pts_c)
    rng = np.random.default_rng(1)
    feats = rng.normal(size=(3, F)).astype(np.float32)
    dd, _, _, _ = oracle.ray(cam, p, 16, 16)
    t = np.float32(3.0)
    # one neighbour -> its own feature
    _, _, fe, _ = oracle.shade(pts, feats, cam, p, dims, mlp, pix, [t], [[1, -1, -1]])
    assert np.allclose(fe[0], feats[1], rtol=1e-12)
    # constant features -> constant
    cf = np.tile(rng.normal(size=(1, F)).astype(np.float32), (3, 1))
    _, _, fe, _ = oracle.shade(pts, cf, cam, p, dims, mlp, pix, [t], [[0, 1, 2]])
    assert np.allclose(fe[0], cf[0], rtol=1e-12)
    # inverse-distance closed form, and invariance to the neighbour order
    x = np.float64(t) * dd.astype(np.float64)
    Pc = oracle.cam_points(cam, pts).astype(np.float64)
    w = 1.0 / np.linalg.norm(x[None] - Pc, axis=1)
    expect = (w[:, None] * feats.astype(np.float64)).sum(0) / w.sum()
    _, _, fe1, _ = oracle.shade(pts, feats, cam, p, dims, mlp, pix, [t], [[0, 1, 2]])
    _, _, fe2, _ = oracle.shade(pts, feats, cam, p, dims, mlp, pix, [t], [[2, 0, 1]])
    assert np.allclose(fe1[0], expect, rtol=1e-12) and np.allclose(fe2[0], fe1[0], rtol=1e-12)


def test_mlp_against_numpy_matmul():
    dims = [32, 128, 128, 128, 4]
    prm = scenes.random_mlp(dims, 3, sigma_bias=2.0)
    x = np.random.default_rng(4).normal(size=32)
    y = oracle.mlp(dims, prm, x)
    h = x
    off = 0
    for l in range(len(dims) - 1):
        fi, fo = dims[l], dims[l + 1]
        W = prm[off: off + fi * fo].astype(np.float64).reshape(fo, fi); off += fi * fo
        bb = prm[off: off + fo].astype(np.float64); off += fo
        h = W @ h + bb
        if l + 1 < len(dims) - 1:
            h = np.maximum(h, 0)
    assert np.allclose(y, h, rtol=1e-12, atol=1e-12)


# ----------------------------------------------------- whole-frame invariants

def test_frame_invariants_small_workload():
    sc = scenes.sphere_plane_64()
    r = oracle.render(sc.points, sc.feats, sc.camera, sc.params, sc.mlp_dims, sc.mlp_params)
    ws, ns, cc = r["wsum"], r["n_s"], r["cand_count"]
    assert np.all(ws >= 0) and np.all(ws <= 1.0)                   # sum of weights <= 1
    assert np.all((ns == 0) == (cc == 0))                            # a hit always yields >= 1 sample
    assert np.all(ns <= sc.params.n_max)
    assert np.all(r["rgb"][ns == 0] == 0.0)                          # black background
    assert np.array_equal(np.diff(r["sample_offset"]), ns)
    assert np.all(r["nbr"][:, 0] >= 0)
    # samples of a ray in depth order, each sample's own point is its nearest neighbour
    for i in np.nonzero(ns > 1)[0][:200]:
        a, b = r["sample_offset"][i], r["sample_offset"][i + 1]
        assert np.all(np.diff(r["t"][a:b]) > 0)
    # the sample's own point lies within its radius, so it is in N_j unless K closer ones fill it
    own = np.array([s_ in row for s_, row in zip(r["src"], r["nbr"])])
    full = np.all(r["nbr"] >= 0, axis=1)
    assert np.all(own | full)
    # primary bucket = key of the first sample's point
    tb = oracle.build_table(sc.points, sc.camera, sc.params)
    keyof = {}
    for k in np.nonzero(np.diff(tb["start"].astype(np.int64)))[0]:
        for i in range(tb["start"][k], tb["start"][k + 1]):
            keyof[int(tb["ids"][i])] = int(k)
    first = r["src"][r["sample_offset"][:-1][ns > 0]]
    assert all(keyof[int(s)] == int(k) for s, k in zip(first, r["primary"][ns > 0]))
    assert np.all(r["primary"][ns == 0] == -1)


def test_frame_permutation_invariance_and_threads():
    pts, feats, cam, p, dims, mlp = tiny_scene(res=16, n=3000, seed=5)
    perm = np.random.default_rng(1).permutation(len(pts))
    a = oracle.render(pts, feats, cam, p, dims, mlp)
    b = oracle.render(pts[perm], feats[perm], cam, p, dims, mlp, nthreads=4)
    for k in ("n_s", "primary", "cand_count", "t", "nbr_dist"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["src"], perm[b["src"]])
    assert np.array_equal(a["rgb"], b["rgb"])


def test_candidate_cap_keeps_nearest():
    pts, feats, cam, p, dims, mlp = tiny_scene(res=16, n=3000, r=0.08)
    full = oracle.render(pts, feats, cam, p, dims, mlp)
    p2 = scenes.Params(**{**p.__dict__, "cand_cap": 4})
    cut = oracle.render(pts, feats, cam, p2, dims, mlp)
    assert np.array_equal(full["cand_count"], cut["cand_count"])     # true counts reported
    assert full["cand_count"].max() > 4
    for pix in np.nonzero(full["cand_count"] > 4)[0][:20]:
        ids, ts, n = oracle.ray_candidates(pts, cam, p, int(pix), brute=False)
        a, b = cut["sample_offset"][pix], cut["sample_offset"][pix + 1]
        assert set(cut["src"][a:b]) <= set(ids[:4])                  # only the 4 nearest in (t, id)
