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
