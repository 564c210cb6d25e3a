"""Pins of the oracle's interval-restricted search with plain fallback
(decision step D12, the search of the learned depth-interval proposal):

* intervals covering [t_near, t_far] reduce it to the plain search;
* on two dense parallel planes, an interval holding only the first plane
  restricts the candidates to that plane (its count is the brute-force count
  of plain candidates inside the interval) and keeps the plain samples;
  intervals that start behind the first plane, or hold no point, fall back
  to the plain search (plain counts and samples)."""
import numpy as np

import oracle
from paper_2404_14044_b300 import scenes

Z1, Z2 = 3.0, 4.5


def _scene():
    cam = scenes.make_camera(24, 24, 30.0, (0.0, -6.0, 0.0), t_near=1.0, t_far=8.0)
    rng = np.random.default_rng(4)
    # two planes y = const facing the camera (depths 3 and 4.5 along the axis)
    n = 6000
    half = 1.6
    p1 = np.stack([rng.uniform(-half, half, n), np.full(n, Z1 - 6.0), rng.uniform(-half, half, n)], 1)
    p2 = np.stack([rng.uniform(-half, half, n), np.full(n, Z2 - 6.0), rng.uniform(-half, half, n)], 1)
    pts = np.concatenate([p1, p2]).astype(np.float32)
    feats = scenes.random_features(len(pts), 8, 1)
    dims = [8, 16, 4]
    mlp = scenes.random_mlp(dims, 2, sigma_bias=30.0)
    p = scenes.Params(r=0.05, K=4, n_max=4)
    return cam, pts, feats, dims, mlp, p


def _render(sc, iv=None):
    cam, pts, feats, dims, mlp, p = sc
    return oracle.render(pts, feats, cam, p, dims, mlp, nthreads=4, intervals=iv)


def _same_samples(a, b, rays):
    for i in rays:
        sa = a["src"][a["sample_offset"][i]:a["sample_offset"][i + 1]]
        sb = b["src"][b["sample_offset"][i]:b["sample_offset"][i + 1]]
        if not np.array_equal(sa, sb):
            return False
    return True


def test_full_range_is_the_plain_search():
    sc = _scene()
    cam = sc[0]
    R = cam.width * cam.height
    plain = _render(sc)
    full = np.tile(np.array([[cam.t_near, cam.t_far]], np.float32), (R, 1))
    res = _render(sc, full)
    for k in ("n_s", "primary", "cand_count", "sample_offset", "t", "src", "nbr", "nbr_dist", "rgb", "wsum"):
        assert np.array_equal(res[k], plain[k]), k


def test_two_planes_restriction_and_fallback():
    sc = _scene()
    cam, pts, feats, dims, mlp, p = sc
    R = cam.width * cam.height
    plain = _render(sc)
    hit = np.nonzero(plain["n_s"] > 0)[0]
    assert len(hit) > 200
    # both planes behind most rays: plain candidates on both
    both = [i for i in hit if plain["cand_count"][i] > 0]
    # (a) the first plane only: restricted candidates, plain samples
    first = np.tile(np.array([[2.0, 3.9]], np.float32), (R, 1))
    ra = _render(sc, first)
    assert _same_samples(ra, plain, hit)
    assert np.array_equal(ra["n_s"], plain["n_s"])
    fewer = 0
    for i in both[::7]:
        ids, ts, n = oracle.ray_candidates(pts, cam, p, int(i), brute=True)
        inside = int(np.sum((ts >= 2.0) & (ts <= np.float32(3.9))))
        assert ra["cand_count"][i] == inside, (i, ra["cand_count"][i], inside)
        fewer += inside < n
    assert fewer > 10
    # (b) starts behind the first plane: the plain search finds points in
    # front of t0, so the ray falls back (plain count and samples)
    behind = np.tile(np.array([[4.0, 5.5]], np.float32), (R, 1))
    rb = _render(sc, behind)
    assert np.array_equal(rb["cand_count"][hit], plain["cand_count"][hit])
    assert _same_samples(rb, plain, hit)
    # (c) an interval with no point in it: empty restricted result, fallback
    empty = np.tile(np.array([[6.5, 7.5]], np.float32), (R, 1))
    rc = _render(sc, empty)
    assert np.array_equal(rc["cand_count"][hit], plain["cand_count"][hit])
    assert np.array_equal(rc["n_s"], plain["n_s"])


def _halo_scene(tn, r, res=120, n_dir=48):
    """Points just inside the radius r of pixel-centre rays at depth tn, in
    n_dir directions perpendicular to each ray, for rays at the image corners,
    edges and centre: the accepted points whose projections lie farthest from
    the ray's pixel, where the D12 window bound is tightest."""
    cam = scenes.make_camera(res, res, 40.0, (0.0, -6.0, 0.0), t_near=1.0, t_far=8.0)
    R = cam.R.astype(np.float64)
    eye = cam.eye()
    pts = []
    rays = []
    for pu in (0, 1, res // 2, res - 2, res - 1):
        for pv in (0, 1, res // 2, res - 2, res - 1):
            d = np.array([(pu + 0.5 - cam.cx) / cam.fx, (pv + 0.5 - cam.cy) / cam.fy, 1.0])
            d /= np.linalg.norm(d)
            a = np.cross(d, [0.0, 0.0, 1.0])
            a /= np.linalg.norm(a)
            b = np.cross(d, a)
            for k in range(n_dir):
                phi = 2 * np.pi * k / n_dir
                for t in (tn * 1.0005, tn * 1.002):
                    pc = t * d + 0.998 * r * (np.cos(phi) * a + np.sin(phi) * b)
                    pts.append(R.T @ pc + eye)
            rays.append(pv * res + pu)
    return cam, np.asarray(pts, np.float32), rays


def test_d12_window_bound_at_its_worst_case():
    # Pinned against brute force where the bound is tightest: points just
    # inside the radius at the interval's start depth, in every direction
    # around corner, edge and centre rays, over a sweep of start depths (so
    # the window's half-width takes several values)
    r = 0.03
    widths = set()
    for tn in np.linspace(1.05, 3.0, 14):
        cam, pts, rays = _halo_scene(float(tn), r)
        p = scenes.Params(r=r, K=4, n_max=4)
        for px in rays:
            b = oracle.ray_candidates_interval(pts, cam, p, px, "brute", np.float32(tn), cam.t_far)
            d = oracle.ray_candidates_interval(pts, cam, p, px, "d12", np.float32(tn), cam.t_far)
            assert b[2] > 0
            assert b[2] == d[2] and np.array_equal(b[0], d[0]), (tn, px, b[2], d[2])
            widths.add(d[3])
    assert len(widths) >= 3, widths


def test_d12_window_holds_every_interval_candidate():
    # The restricted search walks the smaller window D12 derives from the
    # interval's start tn.  Pinned against brute force over all points: for
    # intervals that start just before a ray's first accepted point (the
    # tightest window that point allows) and at random depths, the D12 walk,
    # the full-window walk and brute force return the same candidates.
    rng = np.random.default_rng(12)
    checked = shrunk = 0
    for seed, res in ((0, 96), (1, 120)):
        sc = scenes.objects_800(seed=seed, n_points=60_000, res=res)
        # a radius of several pixels at this resolution, so that h > 1 and the
        # D12 window can shrink
        cam, p = sc.camera, scenes.Params(**{**sc.params.__dict__, "r": 0.03})
        pix = rng.choice(res * res, 400, replace=False)
        for px in pix:
            ids, ts, n, h = oracle.ray_candidates_interval(sc.points, cam, p, int(px), "brute", cam.t_near, cam.t_far)
            if n == 0:
                continue
            t0 = float(ts[0])
            for tn, tf in ((t0 - rng.uniform(0.0, 2.0 * p.r), cam.t_far),
                           (rng.uniform(cam.t_near, t0), t0 + rng.uniform(0.0, 0.2)),
                           (t0 + rng.uniform(0.0, 0.05), cam.t_far)):
                tn, tf = np.float32(max(tn, cam.t_near)), np.float32(min(tf, cam.t_far))
                b = oracle.ray_candidates_interval(sc.points, cam, p, int(px), "brute", tn, tf)
                f = oracle.ray_candidates_interval(sc.points, cam, p, int(px), "full", tn, tf)
                d = oracle.ray_candidates_interval(sc.points, cam, p, int(px), "d12", tn, tf)
                assert b[2] == f[2] == d[2], (px, tn, tf, b[2], f[2], d[2])
                assert np.array_equal(b[0], f[0]) and np.array_equal(b[0], d[0])
                assert np.array_equal(b[1].view(np.int32), d[1].view(np.int32))
                checked += 1
                shrunk += d[3] < f[3]
            if checked >= 150:
                break
    print("checked", checked, "shrunk", shrunk)
    assert checked >= 150 and shrunk >= 50, (checked, shrunk)
