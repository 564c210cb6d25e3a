"""Independent float64 geometry used to pin the oracle: camera transform,
pixel-centre rays, perpendicular distances and the cone radius built from the
similar-triangle construction of the Supplementary (Sec. 1), written from the
geometry rather than from the oracle's float32 formulas."""
import math

import numpy as np


def cam_space(cam, pts):
    R = np.asarray(cam.R, np.float64).reshape(3, 3)
    t = np.asarray(cam.t, np.float64)
    return np.asarray(pts, np.float64) @ R.T + t


def ray_dir(cam, pu, pv):
    v = np.array([(pu + 0.5 - cam.cx) / cam.fx, (pv + 0.5 - cam.cy) / cam.fy, 1.0])
    return v / np.linalg.norm(v)


def perp(P, d):
    """(t, rho) of camera-space points P relative to the ray o=0, unit d."""
    t = P @ d
    e = P - t[:, None] * d[None, :]
    return t, np.linalg.norm(e, axis=1)


def cone_sin(cam, pu, pv, rdd):
    """sin of the angle at the optical centre A between the ray AE (E = pixel
    centre p_o on the f=1 image plane) and AB, with B the point of the
    r-double-dot disc around E nearest the principal point G (the
    construction of the Supplementary).  Eq. radius is t times this."""
    E = np.array([(pu + 0.5 - cam.cx) / cam.fx, (pv + 0.5 - cam.cy) / cam.fy, 1.0])
    G = np.array([0.0, 0.0, 1.0])
    g = G - E
    n = np.linalg.norm(g)
    u = g / n if n > 0 else np.array([1.0, 0.0, 0.0])
    B = E + rdd * u
    c = np.cross(E, B)
    return np.linalg.norm(c) / (np.linalg.norm(E) * np.linalg.norm(B))


def cone_tan_approx(cam, pu, pv, rdd):
    """Small-angle form (Supplementary, AB ~ AF ~ AE): r ~ t rdd f / |p_o - o|^2."""
    E = np.array([(pu + 0.5 - cam.cx) / cam.fx, (pv + 0.5 - cam.cy) / cam.fy, 1.0])
    return rdd / float(E @ E)


def ulp32(x):
    x = np.float32(abs(x))
    return float(np.nextafter(x, np.float32(np.inf)) - x)
