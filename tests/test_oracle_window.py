"""Pin of the depth-bounded plain window (fixed radius).

The search walks a window of half-width h_eff = min(h, floor(lim + 0.5)),
lim = 1.001 win / max(z_min - r sin(theta_max), z_near) + 1e-3, where z_min is
the smallest camera depth of any tabled point: an accepted point lies within
r of the ray point nearest to it, and along that segment (perpendicular to
the ray) the depth falls at most r sin(theta_max) below the point's own.
The window h of the table takes the same bound at t_near cos(theta_max) -
r sin(theta_max).  Here brute force over all points (the oracle's search
without a table) finds every accepted point inside the h_eff window of its
ray, on a scene where h_eff < h."""
import math

import numpy as np

import oracle
from paper_2404_14044_b300 import scenes


def _h_eff(cam, p, h, zmin):
    ax = max(abs(0.5 - cam.cx), abs((cam.width - 0.5) - cam.cx)) / cam.fx
    ay = max(abs(0.5 - cam.cy), abs((cam.height - 0.5) - cam.cy)) / cam.fy
    q = ax * ax + ay * ay
    sin_max = math.sqrt(q / (1.0 + q))
    win = max(cam.fx * p.r * math.sqrt(1.0 + ax * ax), cam.fy * p.r * math.sqrt(1.0 + ay * ay))
    zlo = max(zmin - p.r * sin_max, cam.z_near)
    lim = win / zlo * 1.001 + 1e-3
    return min(h, int(math.floor(lim + 0.5)))


def test_accepted_points_lie_in_the_depth_bounded_window():
    sc = scenes.objects_800(n_points=300_000, res=800)
    cam, p = sc.camera, sc.params
    tab = oracle.build_table(sc.points, cam, p)
    h, start, ids, pos = tab["h"], tab["start"], tab["ids"], tab["pos"]
    zmin = float(pos[:, 2].min())
    he = _h_eff(cam, p, h, zmin)
    assert he < h, (he, h)
    Wp = cam.width + 2 * h
    # padded cell of every tabled point, by original id
    bucket = np.searchsorted(start, np.arange(len(ids)), side="right") - 1
    cell_of = np.full(len(sc.points), -1, np.int64)
    cell_of[ids] = bucket
    rng = np.random.default_rng(3)
    worst, seen = 0, 0
    for pix in rng.integers(0, cam.width * cam.height, 400):
        acc, _, n = oracle.ray_candidates(sc.points, cam, p, int(pix), brute=True)
        if n == 0:
            continue
        pv, pu = divmod(int(pix), cam.width)
        cv, cu = np.divmod(cell_of[acc], Wp)
        assert np.all(cell_of[acc] >= 0)
        off = np.maximum(np.abs(cu - (pu + h)), np.abs(cv - (pv + h)))
        worst = max(worst, int(off.max()))
        seen += n
    assert seen > 1000
    assert worst <= he, (worst, he, h)
