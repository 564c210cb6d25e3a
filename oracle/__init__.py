"""CPU oracle for the HashPoint hot path -- test infrastructure.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It wraps ``hp_oracle.c`` (plain C, double
precision for continuous values, the float32 decision contract for discrete
decisions; see the header comment of that file) through ctypes.  It shares no
code with the CUDA path.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
               "-shared", "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


class Camera(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("R", C.c_float * 9), ("t", C.c_float * 3),
                ("t_near", C.c_float), ("t_far", C.c_float), ("z_near", C.c_float)]


class Params(C.Structure):
    _fields_ = [("radius_mode", C.c_int32), ("r", C.c_float), ("rho", C.c_float), ("gamma", C.c_float),
                ("beta2", C.c_float), ("eps_w", C.c_float), ("gap_k", C.c_float), ("eps_d", C.c_float),
                ("cand_cap", C.c_int32), ("K", C.c_int32), ("n_max", C.c_int32), ("bg_mode", C.c_int32),
                ("window_h", C.c_int32)]


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct)) if a is not None else None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        fp, i32p, u32p, i64p, dp = (C.POINTER(C.c_float), C.POINTER(C.c_int32), C.POINTER(C.c_uint32),
                                    C.POINTER(C.c_int64), C.POINTER(C.c_double))
        L.or_exp32.argtypes = [C.c_float]
        L.or_exp32.restype = C.c_float
        L.or_cam_point.argtypes = [C.POINTER(Camera), fp, fp]
        L.or_cam_points.argtypes = [C.POINTER(Camera), fp, C.c_int64, fp]
        L.or_window.argtypes = [C.POINTER(Camera), C.POINTER(Params), i32p, fp]
        L.or_window.restype = C.c_int
        L.or_build_table.argtypes = [fp, C.c_int64, C.POINTER(Camera), C.c_int32, u32p, i32p, fp]
        L.or_build_table.restype = C.c_int64
        L.or_render.argtypes = [fp, C.c_int64, fp, C.c_int32, C.POINTER(Camera), C.POINTER(Params), i32p,
                                C.c_int32, fp, i32p, C.c_int64, fp, C.c_int32, C.c_int32, i32p, i32p, i32p, i64p,
                                fp, i32p, i32p, i32p, fp, dp, dp, dp, dp]
        L.or_render.restype = C.c_int64
        L.or_ray_candidates.argtypes = [fp, C.c_int64, C.POINTER(Camera), C.POINTER(Params), C.c_int32,
                                        C.c_int32, C.c_int32, i32p, fp]
        L.or_ray_candidates.restype = C.c_int64
        L.or_ray_candidates_interval.argtypes = [fp, C.c_int64, C.POINTER(Camera), C.POINTER(Params), C.c_int32,
                                                 C.c_int32, C.c_float, C.c_float, C.c_int32, i32p, fp, i32p]
        L.or_ray_candidates_interval.restype = C.c_int64
        L.or_shade.argtypes = [fp, fp, C.c_int32, C.POINTER(Camera), C.POINTER(Params), i32p, C.c_int32, fp,
                               C.c_int32, C.c_int32, fp, i32p, dp, dp, dp, dp]
        L.or_mlp.argtypes = [i32p, C.c_int32, fp, dp, dp]
        L.or_ray.argtypes = [C.POINTER(Camera), C.POINTER(Params), C.c_int32, C.c_int32, fp]
        L.or_select.argtypes = [C.POINTER(Camera), C.POINTER(Params), C.c_int32, C.c_int32, fp, i32p, fp, fp,
                                i32p, i32p, fp, i32p, fp, fp]
        L.or_select.restype = C.c_int32
        L.or_backward.argtypes = [fp, C.c_int64, fp, C.c_int32, C.POINTER(Camera), C.POINTER(Params), i32p,
                                  C.c_int32, fp, i32p, C.c_int64, i64p, fp, i32p, i32p, dp, dp, dp, dp, dp]
        L.or_backward.restype = C.c_int64
        L.or_forward_frozen.argtypes = [dp, dp, dp, C.c_int32, C.POINTER(Camera), C.POINTER(Params), i32p,
                                        C.c_int32, fp, i32p, C.c_int64, i64p, fp, i32p, i32p, dp, dp]
        L.or_forward_frozen.restype = C.c_int64
    return _lib


def camera_struct(cam) -> Camera:
    c = Camera()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.R[:] = [float(v) for v in np.asarray(cam.R, np.float32).ravel()]
    c.t[:] = [float(v) for v in np.asarray(cam.t, np.float32).ravel()]
    c.t_near, c.t_far, c.z_near = float(cam.t_near), float(cam.t_far), float(cam.z_near)
    return c


def params_struct(p) -> Params:
    s = Params()
    s.radius_mode, s.r, s.rho = int(p.radius_mode), float(p.r), float(p.rho)
    s.gamma, s.beta2, s.eps_w, s.gap_k, s.eps_d = float(p.gamma), float(p.beta2), float(p.eps_w), float(p.gap_k), float(p.eps_d)
    s.cand_cap, s.K, s.n_max, s.bg_mode, s.window_h = int(p.cand_cap), int(p.K), int(p.n_max), int(p.bg_mode), int(p.window_h)
    return s


def exp32(x: float) -> float:
    return lib().or_exp32(float(x))


def window(cam, params):
    """(h, r_ddot) of the search window, or raises ValueError."""
    h = C.c_int32()
    rdd = C.c_float()
    rc = lib().or_window(C.byref(camera_struct(cam)), C.byref(params_struct(params)), C.byref(h), C.byref(rdd))
    if rc != 0:
        raise ValueError(f"or_window failed ({rc})")
    return h.value, rdd.value


def cam_points(cam, pts: np.ndarray) -> np.ndarray:
    """Camera-space positions under the decision contract (D1)."""
    pts = np.ascontiguousarray(pts, np.float32)
    out = np.empty_like(pts)
    lib().or_cam_points(C.byref(camera_struct(cam)), _p(pts, C.c_float), len(pts), _p(out, C.c_float))
    return out


def build_table(pts: np.ndarray, cam, params):
    h, _ = window(cam, params)
    pts = np.ascontiguousarray(pts, np.float32)
    P = (cam.width + 2 * h) * (cam.height + 2 * h)
    start = np.zeros(P + 1, np.uint32)
    ids = np.zeros(max(len(pts), 1), np.int32)
    pos = np.zeros((max(len(pts), 1), 3), np.float32)
    nv = lib().or_build_table(_p(pts, C.c_float), len(pts), C.byref(camera_struct(cam)), h,
                              _p(start, C.c_uint32), _p(ids, C.c_int32), _p(pos, C.c_float))
    return dict(h=h, start=start, ids=ids[:nv].copy(), pos=pos[:nv].copy(), n_visible=int(nv))


def ray_candidates(pts, cam, params, pixel: int, brute: bool, cap: int = 4096):
    pts = np.ascontiguousarray(pts, np.float32)
    cid = np.zeros(cap, np.int32)
    ct = np.zeros(cap, np.float32)
    n = lib().or_ray_candidates(_p(pts, C.c_float), len(pts), C.byref(camera_struct(cam)),
                                C.byref(params_struct(params)), int(pixel), int(brute), cap,
                                _p(cid, C.c_int32), _p(ct, C.c_float))
    if n < 0:
        raise ValueError(f"or_ray_candidates failed ({n})")
    return cid[: min(n, cap)].copy(), ct[: min(n, cap)].copy(), int(n)


def render(pts, feats, cam, params, mlp_dims, mlp_params, rays=None, brute=False, nthreads=1,
           per_sample=False, intervals=None):
    """Run the whole frame.  Returns a dict of numpy arrays (see or_render).
    ``intervals`` (R x 2 float32): per-ray depth restriction with the plain
    search as the fallback for rays it leaves empty."""
    iv = None if intervals is None else np.ascontiguousarray(intervals, np.float32)
    pts = np.ascontiguousarray(pts, np.float32)
    feats = np.ascontiguousarray(feats, np.float32)
    F = feats.shape[1]
    dims = np.ascontiguousarray(mlp_dims, np.int32)
    mlp = np.ascontiguousarray(mlp_params, np.float32)
    R = cam.width * cam.height if rays is None else len(rays)
    rays_a = None if rays is None else np.ascontiguousarray(rays, np.int32)
    K, n_max = params.K, params.n_max
    cap = max(R * n_max, 1)
    out = dict(
        n_s=np.zeros(max(R, 1), np.int32), primary=np.zeros(max(R, 1), np.int32),
        cand_count=np.zeros(max(R, 1), np.int32), sample_offset=np.zeros(R + 1, np.int64),
        t=np.zeros(cap, np.float32), ray=np.zeros(cap, np.int32), src=np.zeros(cap, np.int32),
        nbr=np.zeros(cap * K, np.int32), nbr_dist=np.zeros(cap * K, np.float32),
        rgb=np.zeros(max(R, 1) * 3, np.float64), wsum=np.zeros(max(R, 1), np.float64))
    feat_o = np.zeros(cap * F, np.float64) if per_sample else None
    out4 = np.zeros(cap * 4, np.float64) if per_sample else None
    S = lib().or_render(
        _p(pts, C.c_float), len(pts), _p(feats, C.c_float), F, C.byref(camera_struct(cam)),
        C.byref(params_struct(params)), _p(dims, C.c_int32), len(dims) - 1, _p(mlp, C.c_float),
        _p(rays_a, C.c_int32), R, _p(iv, C.c_float), int(brute), int(nthreads),
        _p(out["n_s"], C.c_int32), _p(out["primary"], C.c_int32), _p(out["cand_count"], C.c_int32),
        _p(out["sample_offset"], C.c_int64), _p(out["t"], C.c_float), _p(out["ray"], C.c_int32),
        _p(out["src"], C.c_int32), _p(out["nbr"], C.c_int32), _p(out["nbr_dist"], C.c_float),
        _p(out["rgb"], C.c_double), _p(out["wsum"], C.c_double), _p(feat_o, C.c_double), _p(out4, C.c_double))
    if S < 0:
        raise ValueError(f"or_render failed ({S})")
    res = dict(S=int(S), n_s=out["n_s"][:R], primary=out["primary"][:R], cand_count=out["cand_count"][:R],
               sample_offset=out["sample_offset"], t=out["t"][:S], ray=out["ray"][:S], src=out["src"][:S],
               nbr=out["nbr"][: S * K].reshape(S, K), nbr_dist=out["nbr_dist"][: S * K].reshape(S, K),
               rgb=out["rgb"][: R * 3].reshape(R, 3), wsum=out["wsum"][:R])
    if per_sample:
        res["feat"] = feat_o[: S * F].reshape(S, F)
        res["out4"] = out4[: S * 4].reshape(S, 4)
    return res


def ray_candidates_interval(pts, cam, params, pixel: int, mode: str, tn: float, tf: float, cap: int = 4096):
    """Accepted points of one ray with t in [tn, tf]: ``mode`` "brute" (all
    points), "full" (the hashed walk of the whole window h) or "d12" (the
    hashed walk of the window the restricted search derives from tn).
    Returns (ids, ts, count, window half-width walked)."""
    pts = np.ascontiguousarray(pts, np.float32)
    cid = np.zeros(cap, np.int32)
    ct = np.zeros(cap, np.float32)
    hw = np.zeros(1, np.int32)
    m = {"brute": 0, "full": 1, "d12": 2}[mode]
    n = lib().or_ray_candidates_interval(_p(pts, C.c_float), len(pts), C.byref(camera_struct(cam)),
                                         C.byref(params_struct(params)), int(pixel), m, float(tn), float(tf), cap,
                                         _p(cid, C.c_int32), _p(ct, C.c_float), _p(hw, C.c_int32))
    if n < 0:
        raise ValueError(f"or_ray_candidates_interval failed ({n})")
    return cid[: min(n, cap)].copy(), ct[: min(n, cap)].copy(), int(n), int(hw[0])


def shade(pts, feats, cam, params, mlp_dims, mlp_params, pixel, ts, nbr):
    """Continuous stages (Sec. 3.4, Eq. 2) for caller-given samples of one ray."""
    pts = np.ascontiguousarray(pts, np.float32)
    feats = np.ascontiguousarray(feats, np.float32)
    F = feats.shape[1]
    dims = np.ascontiguousarray(mlp_dims, np.int32)
    mlp = np.ascontiguousarray(mlp_params, np.float32)
    ts = np.ascontiguousarray(ts, np.float32)
    nbr = np.ascontiguousarray(nbr, np.int32).reshape(len(ts), params.K)
    rgb = np.zeros(3)
    ws = np.zeros(1)
    fo = np.zeros(max(len(ts), 1) * F)
    o4 = np.zeros(max(len(ts), 1) * 4)
    lib().or_shade(_p(pts, C.c_float), _p(feats, C.c_float), F, C.byref(camera_struct(cam)),
                   C.byref(params_struct(params)), _p(dims, C.c_int32), len(dims) - 1, _p(mlp, C.c_float),
                   int(pixel), len(ts), _p(ts, C.c_float), _p(nbr, C.c_int32), _p(rgb, C.c_double),
                   _p(ws, C.c_double), _p(fo, C.c_double), _p(o4, C.c_double))
    return rgb, float(ws[0]), fo[: len(ts) * F].reshape(len(ts), F), o4[: len(ts) * 4].reshape(len(ts), 4)


def mlp(mlp_dims, mlp_params, x: np.ndarray) -> np.ndarray:
    dims = np.ascontiguousarray(mlp_dims, np.int32)
    prm = np.ascontiguousarray(mlp_params, np.float32)
    x = np.ascontiguousarray(x, np.float64)
    y = np.zeros(dims[-1])
    lib().or_mlp(_p(dims, C.c_int32), len(dims) - 1, _p(prm, C.c_float), _p(x, C.c_double), _p(y, C.c_double))
    return y


def ray(cam, params, pu: int, pv: int):
    """(d[3], n2, len, c) of pixel (pu, pv) under D3/D4."""
    o = np.zeros(6, np.float32)
    lib().or_ray(C.byref(camera_struct(cam)), C.byref(params_struct(params)), int(pu), int(pv), _p(o, C.c_float))
    return o[:3].copy(), float(o[3]), float(o[4]), float(o[5])


def select(cam, params, pixel, t, ids, P):
    """Selection (Sec. 3.3) on caller-given candidates of one ray."""
    t = np.ascontiguousarray(t, np.float32)
    ids = np.ascontiguousarray(ids, np.int32)
    P = np.ascontiguousarray(P, np.float32).reshape(-1, 3)
    Cn = len(t)
    n, K = params.n_max, params.K
    ot = np.zeros(n, np.float32)
    osrc = np.zeros(n, np.int32)
    onbr = np.zeros(n * K, np.int32)
    od = np.zeros(n * K, np.float32)
    js = C.c_int32()
    dj = np.zeros(max(Cn, 1), np.float32)
    wj = np.zeros(max(Cn, 1), np.float32)
    ns = lib().or_select(C.byref(camera_struct(cam)), C.byref(params_struct(params)), int(pixel), Cn,
                         _p(t, C.c_float), _p(ids, C.c_int32), _p(P, C.c_float), _p(ot, C.c_float),
                         _p(osrc, C.c_int32), _p(onbr, C.c_int32), _p(od, C.c_float), C.byref(js),
                         _p(dj, C.c_float), _p(wj, C.c_float))
    return dict(n_s=int(ns), t=ot[:ns], src=osrc[:ns], nbr=onbr[: ns * K].reshape(ns, K),
                nbr_dist=od[: ns * K].reshape(ns, K), jstar=int(js.value), d=dj[:Cn], w=wj[:Cn])


def backward(pts, feats, cam, params, mlp_dims, mlp_params, frame, grad_rgb, grad_wsum=None, rays=None):
    """Gradients of the frame ``frame`` (an or_render result) with respect to
    the features and positions, for output gradients grad_rgb (R x 3) and
    grad_wsum (R).  Returns (g_feats N x F, g_pcam N x 3, g_pworld N x 3), double."""
    pts = np.ascontiguousarray(pts, np.float32)
    feats = np.ascontiguousarray(feats, np.float32)
    N, F = feats.shape
    R = len(frame["n_s"])
    dims = np.ascontiguousarray(mlp_dims, np.int32)
    mlp = np.ascontiguousarray(mlp_params, np.float32)
    rays_a = None if rays is None else np.ascontiguousarray(rays, np.int32)
    gr = np.ascontiguousarray(grad_rgb, np.float64).reshape(R, 3)
    gw = None if grad_wsum is None else np.ascontiguousarray(grad_wsum, np.float64)
    gf = np.zeros((max(N, 1), F))
    gpc = np.zeros((max(N, 1), 3))
    gpw = np.zeros((max(N, 1), 3))
    off = np.ascontiguousarray(frame["sample_offset"], np.int64)
    st = np.ascontiguousarray(frame["t"], np.float32)
    ss = np.ascontiguousarray(frame["src"], np.int32)
    sn = np.ascontiguousarray(frame["nbr"], np.int32)
    rc = lib().or_backward(_p(pts, C.c_float), N, _p(feats, C.c_float), F, C.byref(camera_struct(cam)),
                           C.byref(params_struct(params)), _p(dims, C.c_int32), len(dims) - 1, _p(mlp, C.c_float),
                           _p(rays_a, C.c_int32), R, _p(off, C.c_int64), _p(st, C.c_float), _p(ss, C.c_int32),
                           _p(sn, C.c_int32), _p(gr, C.c_double), _p(gw, C.c_double), _p(gf, C.c_double),
                           _p(gpc, C.c_double), _p(gpw, C.c_double))
    if rc != 0:
        raise ValueError(f"or_backward failed ({rc})")
    return gf[:N], gpc[:N], gpw[:N]


def forward_frozen(pcam, pcam0, feats, cam, params, mlp_dims, mlp_params, frame, rays=None):
    """rgb (R x 3), wsum (R) of the frame with its discrete structure frozen,
    at camera-space positions pcam (double) and features feats (double)."""
    pcam = np.ascontiguousarray(pcam, np.float64)
    pcam0 = np.ascontiguousarray(pcam0, np.float64)
    feats = np.ascontiguousarray(feats, np.float64)
    F = feats.shape[1]
    R = len(frame["n_s"])
    dims = np.ascontiguousarray(mlp_dims, np.int32)
    mlp = np.ascontiguousarray(mlp_params, np.float32)
    rays_a = None if rays is None else np.ascontiguousarray(rays, np.int32)
    rgb = np.zeros((max(R, 1), 3))
    ws = np.zeros(max(R, 1))
    off = np.ascontiguousarray(frame["sample_offset"], np.int64)
    st = np.ascontiguousarray(frame["t"], np.float32)
    ss = np.ascontiguousarray(frame["src"], np.int32)
    sn = np.ascontiguousarray(frame["nbr"], np.int32)
    rc = lib().or_forward_frozen(_p(pcam, C.c_double), _p(pcam0, C.c_double), _p(feats, C.c_double), F,
                                 C.byref(camera_struct(cam)), C.byref(params_struct(params)), _p(dims, C.c_int32),
                                 len(dims) - 1, _p(mlp, C.c_float), _p(rays_a, C.c_int32), R, _p(off, C.c_int64),
                                 _p(st, C.c_float), _p(ss, C.c_int32), _p(sn, C.c_int32), _p(rgb, C.c_double),
                                 _p(ws, C.c_double))
    if rc != 0:
        raise ValueError(f"or_forward_frozen failed ({rc})")
    return rgb[:R], ws[:R]
