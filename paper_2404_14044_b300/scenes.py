"""Seeded synthetic inputs for the HashPoint hot path.

This module only *generates inputs*: point clouds, cameras, per-point
features, radiance-MLP weights and ray lists.  It holds none of the method's
arithmetic (no projection, search, selection, aggregation or compositing), so
the CUDA path and the CPU oracle can both take their inputs from it without
sharing any of the computation they are compared on.

Everything is drawn in float64 from ``numpy.random.default_rng(seed)`` and
stored as float32 (C-contiguous), as the C-ABI expects.

Workloads (shapes of the paper's benchmarks, no dataset contents):

* ``sphere_plane_64``  – 64x64 image, fov 40 deg, camera 3 units from the
  origin; 20k points: half area-uniform on the unit sphere, half uniform on
  the plane z=-1 over [-2,2]^2; r=0.02, K=8, n=4, MLP 32-64-64-4.
* ``objects_800``      – 800x800 image, fov 40 deg, camera on a radius-4
  sphere looking at the origin (near 2 / far 6 bounds, the Synthetic-NeRF
  object-centric set-up of Sec. 4); 1M points area-uniform on 6
  nested/overlapping closed shapes (ellipsoids, boxes, tori); r=0.005,
  K=8, n=8, MLP 32-128-128-128-4.
* ``forward_1008``     – 1008x756 forward-facing image (fx=fy=0.8*1008);
  1.5M points: 1.2M on a 4-layer random height field and 0.3M on 50 small
  occluder patches in front of it, normals near +z; cone radius (Eq. radius,
  r-double-dot / r-dot = 2, i.e. kernel size s=5), K=16, n=8.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

# Radius modes (the boundary's hp_config.radius_mode)
RADIUS_FIXED = 0
RADIUS_CONE_EXACT = 1
RADIUS_CONE_APPROX = 2


@dataclasses.dataclass
class Camera:
    """Pinhole camera, world->camera rigid transform (OpenCV axes: x right,
    y down, z forward).  ``R`` is row-major 3x3 float32, ``t`` float32[3]."""

    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    R: np.ndarray
    t: np.ndarray
    t_near: float
    t_far: float
    z_near: float

    def eye(self) -> np.ndarray:
        """Camera centre in world coordinates (float64)."""
        R = self.R.astype(np.float64)
        return -R.T @ self.t.astype(np.float64)


@dataclasses.dataclass
class Params:
    """Method hyper-parameters (Sec. 3.2-3.3 plus the readings of the
    ambiguous points).  Mirrors hp_config of the C-ABI."""

    radius_mode: int = RADIUS_FIXED
    r: float = 0.005             # fixed search radius / r_min for the cone
    rho: float = 0.0             # r_ddot / r_dot (cone modes); <=0: derive from r
    gamma: float = 0.9           # alpha = gamma * exp(-d^2 / beta^2)
    beta2: float = 0.02          # beta^2 (Fig. noisy_input caption default)
    eps_w: float = 1e-3          # keep candidates with w_j > eps_w
    gap_k: float = 4.0           # primary cluster: t-gap <= gap_k * r(t)
    eps_d: float = 1e-6          # IDW distance floor
    cand_cap: int = 128          # candidate list capacity per ray
    K: int = 8                   # neighbours per candidate (pseudo-UDF, IDW)
    n_max: int = 8               # max samples per ray
    bg_mode: int = 0             # 0 black background, 1 white
    window_h: int = 0            # 0: derive the window half-width


@dataclasses.dataclass
class Scene:
    name: str
    points: np.ndarray           # (N,3) float32 world positions
    feats: np.ndarray            # (N,F) float32 point features
    camera: Camera
    params: Params
    mlp_dims: List[int]
    mlp_params: np.ndarray       # packed float32: W0,b0,W1,b1,...  (W row-major out x in)

    @property
    def n_rays_full(self) -> int:
        return self.camera.width * self.camera.height


# ----------------------------------------------------------------- cameras

def intrinsics_from_fov(width: int, height: int, fov_deg: float) -> Tuple[float, float, float, float]:
    """Square pixels, horizontal field of view ``fov_deg``, principal point at
    the image centre."""
    f = (width / 2.0) / math.tan(math.radians(fov_deg) / 2.0)
    return f, f, width / 2.0, height / 2.0


def look_at(eye, target=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0)) -> Tuple[np.ndarray, np.ndarray]:
    """World->camera (R, t) for a camera at ``eye`` looking at ``target``.
    Camera axes: x right, y down, z forward."""
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    up = np.asarray(up, np.float64)
    if abs(float(np.dot(fwd, up))) > 0.999:
        up = np.array([0.0, 1.0, 0.0])
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd], 0)
    t = -R @ eye
    return R.astype(np.float32), t.astype(np.float32)


def make_camera(width, height, fov_deg, eye, t_near, t_far, z_near=0.05, target=(0, 0, 0), up=(0, 0, 1)) -> Camera:
    fx, fy, cx, cy = intrinsics_from_fov(width, height, fov_deg)
    R, t = look_at(eye, target, up)
    return Camera(width, height, float(fx), float(fy), float(cx), float(cy), R, t,
                  float(t_near), float(t_far), float(z_near))


def random_sphere_cameras(n: int, radius: float, seed: int, width=800, height=800, fov_deg=40.0,
                          t_near=2.0, t_far=6.0) -> List[Camera]:
    """``n`` cameras uniform on a sphere of ``radius`` looking at the origin."""
    rng = np.random.default_rng(seed)
    cams = []
    for _ in range(n):
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        cams.append(make_camera(width, height, fov_deg, radius * v, t_near, t_far))
    return cams


# ------------------------------------------------------------ shape sampling

def _unit_sphere(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _random_rotation(rng) -> np.ndarray:
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def sample_ellipsoid(rng, n, axes):
    """Area-uniform samples on an ellipsoid with semi-axes ``axes`` (rejection
    on the area element of the map from the unit sphere)."""
    a, b, c = axes
    gmax = max(b * c, a * c, a * b)
    out = []
    got = 0
    while got < n:
        u = _unit_sphere(rng, 2 * (n - got) + 64)
        g = np.sqrt((b * c * u[:, 0]) ** 2 + (a * c * u[:, 1]) ** 2 + (a * b * u[:, 2]) ** 2)
        keep = rng.random(len(u)) * gmax < g
        u = u[keep][: n - got]
        out.append(u * np.array([a, b, c]))
        got += len(u)
    return np.concatenate(out, 0)


def ellipsoid_area(axes, rng=None) -> float:
    rng = rng or np.random.default_rng(12345)
    a, b, c = axes
    u = _unit_sphere(rng, 200000)
    g = np.sqrt((b * c * u[:, 0]) ** 2 + (a * c * u[:, 1]) ** 2 + (a * b * u[:, 2]) ** 2)
    return float(4 * math.pi * g.mean())


def sample_box(rng, n, half):
    """Area-uniform samples on the surface of an axis-aligned box."""
    hx, hy, hz = half
    areas = np.array([hy * hz, hy * hz, hx * hz, hx * hz, hx * hy, hx * hy])
    face = rng.choice(6, size=n, p=areas / areas.sum())
    s = rng.uniform(-1, 1, size=(n, 2))
    p = np.zeros((n, 3))
    for f in range(6):
        m = face == f
        axis, sign = f // 2, (1.0 if f % 2 == 0 else -1.0)
        others = [i for i in range(3) if i != axis]
        p[m, axis] = sign * half[axis]
        p[m, others[0]] = s[m, 0] * half[others[0]]
        p[m, others[1]] = s[m, 1] * half[others[1]]
    return p


def box_area(half) -> float:
    hx, hy, hz = half
    return 8.0 * (hx * hy + hy * hz + hx * hz)


def sample_torus(rng, n, R, r):
    """Area-uniform samples on a torus (rejection on R + r cos v)."""
    out = []
    got = 0
    while got < n:
        m = 2 * (n - got) + 64
        u = rng.uniform(0, 2 * math.pi, m)
        v = rng.uniform(0, 2 * math.pi, m)
        keep = rng.random(m) * (R + r) < (R + r * np.cos(v))
        u, v = u[keep][: n - got], v[keep][: n - got]
        out.append(np.stack([(R + r * np.cos(v)) * np.cos(u), (R + r * np.cos(v)) * np.sin(u), r * np.sin(v)], 1))
        got += len(u)
    return np.concatenate(out, 0)


def torus_area(R, r) -> float:
    return 4.0 * math.pi * math.pi * R * r


def _split_counts(n, weights):
    w = np.asarray(weights, np.float64)
    w = w / w.sum()
    c = np.floor(w * n).astype(np.int64)
    rem = n - int(c.sum())
    order = np.argsort(-(w * n - c))
    c[order[:rem]] += 1
    return c


def object_points(n_points: int, seed: int, n_shapes: int = 6) -> np.ndarray:
    """``n_points`` area-uniform points on ``n_shapes`` nested/overlapping
    closed shapes with centres in [-0.5,0.5]^3 (ellipsoids, boxes, tori in
    turn).  Sizes are chosen so the scene stays inside the radius-2 ball that
    the near=2 / far=6 bounds of a radius-4 camera enclose."""
    rng = np.random.default_rng(seed)
    shapes = []
    for i in range(n_shapes):
        centre = rng.uniform(-0.5, 0.5, 3)
        rot = _random_rotation(rng)
        kind = i % 3
        if kind == 0:
            axes = rng.uniform(0.3, 1.0, 3)
            shapes.append(("ellipsoid", centre, rot, axes, ellipsoid_area(axes)))
        elif kind == 1:
            half = rng.uniform(0.2, 0.6, 3)
            shapes.append(("box", centre, rot, half, box_area(half)))
        else:
            R_, r_ = rng.uniform(0.4, 0.8), rng.uniform(0.1, 0.25)
            shapes.append(("torus", centre, rot, (R_, r_), torus_area(R_, r_)))
    counts = _split_counts(n_points, [s[4] for s in shapes])
    pts = []
    for (kind, centre, rot, prm, _), c in zip(shapes, counts):
        if kind == "ellipsoid":
            p = sample_ellipsoid(rng, int(c), prm)
        elif kind == "box":
            p = sample_box(rng, int(c), prm)
        else:
            p = sample_torus(rng, int(c), *prm)
        pts.append(p @ rot.T + centre)
    pts = np.concatenate(pts, 0)
    pts = pts[rng.permutation(len(pts))]
    return np.ascontiguousarray(pts.astype(np.float32))


def sphere_plane_points(n_sphere: int, n_plane: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    s = _unit_sphere(rng, n_sphere)
    pl = np.stack([rng.uniform(-2, 2, n_plane), rng.uniform(-2, 2, n_plane), -np.ones(n_plane)], 1)
    pts = np.concatenate([s, pl], 0)
    pts = pts[rng.permutation(len(pts))]
    return np.ascontiguousarray(pts.astype(np.float32))


def forward_points(n_field: int, n_occ: int, seed: int, width=1008, height=756, f=806.4,
                   n_layers=4, n_patches=50) -> np.ndarray:
    """Forward-facing scene seen by a camera at the origin looking along +z:
    ``n_layers`` random height fields z = z_k + 0.1*noise(x,y) at depths
    2,3,4,5 covering the frustum, and ``n_patches`` small planar occluder
    patches at depths 1..2 whose normals are +z perturbed by N(0,0.1)."""
    rng = np.random.default_rng(seed)
    hx, hy = (width / 2) / f, (height / 2) / f       # tan of the half-fovs
    counts = _split_counts(n_field, [(2 + k) ** 2 for k in range(n_layers)])
    pts = []
    for k in range(n_layers):
        z0 = 2.0 + k
        c = int(counts[k])
        x = rng.uniform(-1.1 * hx * z0, 1.1 * hx * z0, c)
        y = rng.uniform(-1.1 * hy * z0, 1.1 * hy * z0, c)
        # smooth noise: a few random sinusoids
        noise = np.zeros(c)
        for _ in range(4):
            kx, ky = rng.normal(0, 3.0, 2)
            ph = rng.uniform(0, 2 * math.pi)
            noise += np.sin(kx * x + ky * y + ph) / 4.0
        pts.append(np.stack([x, y, z0 + 0.1 * noise], 1))
    per = _split_counts(n_occ, np.ones(n_patches))
    for p in range(n_patches):
        z0 = rng.uniform(1.0, 2.0)
        cx_, cy_ = rng.uniform(-hx * z0, hx * z0), rng.uniform(-hy * z0, hy * z0)
        size = rng.uniform(0.05, 0.2)
        nrm = np.array([0.0, 0.0, -1.0]) + rng.normal(0, 0.1, 3)
        nrm /= np.linalg.norm(nrm)
        a = np.cross(nrm, [1.0, 0.0, 0.0])
        a /= np.linalg.norm(a)
        b = np.cross(nrm, a)
        s = rng.uniform(-size, size, (int(per[p]), 2))
        pts.append(np.array([cx_, cy_, z0]) + s[:, :1] * a + s[:, 1:] * b)
    pts = np.concatenate(pts, 0)
    pts = pts[rng.permutation(len(pts))]
    return np.ascontiguousarray(pts.astype(np.float32))


# --------------------------------------------------------- features, MLP, rays

def random_features(n: int, F: int, seed: int, std: float = 0.1) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.normal(0.0, std, (n, F)).astype(np.float32))


def random_mlp(dims: List[int], seed: int, sigma_bias: float = 0.0) -> np.ndarray:
    """He-uniform weights, zero biases except the density output (channel 0
    of the last layer), packed W0,b0,W1,b1,... with W row-major (out x in)."""
    rng = np.random.default_rng(seed)
    parts = []
    for l in range(len(dims) - 1):
        fi, fo = dims[l], dims[l + 1]
        lim = math.sqrt(6.0 / fi)
        W = rng.uniform(-lim, lim, (fo, fi))
        b = np.zeros(fo)
        if l == len(dims) - 2:
            b[0] = sigma_bias
        parts += [W.ravel(), b]
    return np.ascontiguousarray(np.concatenate(parts).astype(np.float32))


def proposal_params(seed: int, out_bias=(-3.0, 3.0), scale: float = 1.0) -> np.ndarray:
    """Parameters of the 16-32-32-2 depth-interval network in the packed
    layout above (He-uniform weights times ``scale``, zero hidden biases);
    the output biases start the interval wide (t0 near t_near, t1 near
    t_far) by default."""
    th = random_mlp([16, 32, 32, 2], seed).astype(np.float64) * scale
    th[-2:] = out_bias
    out = th.astype(np.float32)
    assert out.size == 1666
    return out


def mlp_param_count(dims: List[int]) -> int:
    return sum(dims[l] * dims[l + 1] + dims[l + 1] for l in range(len(dims) - 1))


def random_rays(width: int, height: int, n: int, seed: int) -> np.ndarray:
    """``n`` distinct random pixel ids (row-major v*width+u), int32."""
    rng = np.random.default_rng(seed)
    ids = rng.choice(width * height, size=n, replace=False)
    return np.ascontiguousarray(ids.astype(np.int32))


# ------------------------------------------------------------ named workloads

def sphere_plane_64(seed: int = 0, n_sphere: int = 10000, n_plane: int = 10000, res: int = 64) -> Scene:
    cam = make_camera(res, res, 40.0, (0.0, -3.0, 0.0), t_near=1.0, t_far=10.0)
    pts = sphere_plane_points(n_sphere, n_plane, seed)
    params = Params(radius_mode=RADIUS_FIXED, r=0.02, K=8, n_max=4)
    dims = [32, 64, 64, 4]
    return Scene("sphere_plane_64", pts, random_features(len(pts), 32, seed + 1), cam, params, dims,
                 random_mlp(dims, seed, sigma_bias=1.5 / params.r))


def objects_800(seed: int = 0, n_points: int = 1_000_000, res: int = 800, view: int = 0) -> Scene:
    cam = random_sphere_cameras(view + 1, 4.0, seed, width=res, height=res)[view]
    pts = object_points(n_points, seed)
    params = Params(radius_mode=RADIUS_FIXED, r=0.005, K=8, n_max=8)
    dims = [32, 128, 128, 128, 4]
    return Scene("objects_800", pts, random_features(len(pts), 32, seed + 1), cam, params, dims,
                 random_mlp(dims, seed, sigma_bias=1.5 / params.r))


def forward_1008(seed: int = 0, n_field: int = 1_200_000, n_occ: int = 300_000, width: int = 1008,
                 height: int = 756, mode: int = RADIUS_CONE_EXACT) -> Scene:
    f = 0.8 * width
    cam = Camera(width, height, f, f, width / 2.0, height / 2.0, np.eye(3, dtype=np.float32),
                 np.zeros(3, np.float32), 0.5, 10.0, 0.05)
    pts = forward_points(n_field, n_occ, seed, width, height, f)
    params = Params(radius_mode=mode, r=0.0, rho=2.0, K=16, n_max=8)
    dims = [32, 128, 128, 128, 4]
    # cone radius at depth ~3: 3 * rho * sqrt(1/(pi f^2)) ~ 0.004
    return Scene("forward_1008", pts, random_features(len(pts), 32, seed + 1), cam, params, dims,
                 random_mlp(dims, seed, sigma_bias=1.5 / 0.004))


def forward_cameras(n: int, seed: int, width: int = 1008, height: int = 756, max_shift: float = 0.15,
                    max_angle_deg: float = 3.0) -> List[Camera]:
    """Forward-facing views of the ``forward_1008`` scene: the reference
    camera (at the origin, looking +z) moved by up to ``max_shift`` along each
    axis and turned by up to ``max_angle_deg`` about x and y, as in a
    hand-held forward-facing capture.  View 0 is the reference camera."""
    rng = np.random.default_rng(seed)
    f = 0.8 * width
    cams = []
    for i in range(n):
        if i == 0:
            R = np.eye(3)
            eye = np.zeros(3)
        else:
            ax, ay = np.radians(rng.uniform(-max_angle_deg, max_angle_deg, 2))
            Rx = np.array([[1, 0, 0], [0, math.cos(ax), -math.sin(ax)], [0, math.sin(ax), math.cos(ax)]])
            Ry = np.array([[math.cos(ay), 0, math.sin(ay)], [0, 1, 0], [-math.sin(ay), 0, math.cos(ay)]])
            R = Rx @ Ry                       # world -> camera rotation
            eye = rng.uniform(-max_shift, max_shift, 3)
        t = -R @ eye
        cams.append(Camera(width, height, f, f, width / 2.0, height / 2.0, R.astype(np.float32),
                           t.astype(np.float32), 0.5, 10.0, 0.05))
    return cams


WORKLOADS = {
    "sphere_plane_64": sphere_plane_64,
    "objects_800": objects_800,
    "forward_1008": forward_1008,
}
