"""Python binding of the C-ABI library ``libhashpoint.so`` (argument
marshalling only: every step of the hot path runs in the library's CUDA
kernels).  PyTorch provides device memory and streams.

The library must have been built (``python -m paper_2404_14044_b300.build``);
importing the binding without it raises ``RuntimeError`` -- there is no
fallback path.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import json
import os
import struct
from typing import Dict, Optional, Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhashpoint.so")

HP_OK, HP_ERR_INVALID_ARG, HP_ERR_CUDA, HP_ERR_OVERFLOW, HP_ERR_TIMEOUT = 0, 1, 2, 3, 4
HP_ERR_NOT_BUILT, HP_ERR_NO_MEMORY, HP_ERR_BAD_RAY, HP_ERR_TOO_LARGE, HP_ERR_BOUNDS = 5, 6, 7, 8, 9
SCAN_NOALLOC_MAX_N = 67108864
MLP_MAX_LAYERS = 8

# every symbol include/hashpoint.h declares
SYMBOLS = ("hp_create", "hp_destroy", "hp_workspace_size", "hp_window", "hp_set_workspace", "hp_build_table",
           "hp_table_info", "hp_table_copy", "hp_search_sample", "hp_aggregate_render",
           "hp_aggregate_render_backward", "hp_get_status",
           "hp_debug_fault", "hp_profile_start", "hp_profile_stop", "hp_profile_kernel_name",
           "hp_selftest_mma", "hp_scan_noalloc", "hp_proposal_infer", "hp_proposal_train_step",
           "hp_search_sample_proposal", "hp_search_sample_learned", "hp_status_string", "hp_version")
PROF_KERNELS = 15
PROP_PARAMS = 1666
PROP_BINS = 16


class HPError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {status_string(code)} ({code})")
        self.code = code


class Camera(C.Structure):
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("R", C.c_float * 9), ("t", C.c_float * 3),
                ("t_near", C.c_float), ("t_far", C.c_float), ("z_near", C.c_float)]


class Config(C.Structure):
    _fields_ = [("radius_mode", C.c_int32), ("rho", C.c_float), ("gamma", C.c_float), ("beta2", C.c_float),
                ("eps_w", C.c_float), ("gap_k", C.c_float), ("eps_d", C.c_float), ("cand_cap", C.c_int32),
                ("bg_mode", C.c_int32), ("window_h", C.c_int32)]


class Samples(C.Structure):
    _fields_ = [("n_s", C.c_void_p), ("primary", C.c_void_p), ("cand_count", C.c_void_p),
                ("sample_offset", C.c_void_p), ("t", C.c_void_p), ("ray", C.c_void_p), ("src", C.c_void_p),
                ("delta", C.c_void_p), ("nbr", C.c_void_p), ("nbr_dist", C.c_void_p), ("capacity", C.c_int64)]


class Mlp(C.Structure):
    _fields_ = [("n_layers", C.c_int32), ("dims", C.c_int32 * (MLP_MAX_LAYERS + 1)), ("d_params", C.c_void_p),
                ("decode", C.c_int32)]


DECODE_FP32, DECODE_FP32_SIMT, DECODE_BF16 = 0, 1, 2


class Table(C.Structure):
    _fields_ = [("h", C.c_int32), ("padded_width", C.c_int32), ("padded_height", C.c_int32),
                ("n_buckets", C.c_int64), ("r_ddot", C.c_float), ("d_start", C.c_void_p), ("d_points", C.c_void_p)]


_lib = None


def lib():
    """Load libhashpoint.so (raises RuntimeError if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2404_14044_b300.build`")
        L = C.CDLL(LIB_PATH)
        vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int32
        L.hp_create.argtypes = [C.POINTER(vp), C.POINTER(Config)]
        L.hp_destroy.argtypes = [vp]
        L.hp_workspace_size.argtypes = [C.POINTER(Config), C.POINTER(Camera), C.c_float, i64, i64, i32, i32,
                                        C.POINTER(C.c_size_t)]
        L.hp_window.argtypes = [C.POINTER(Config), C.POINTER(Camera), C.c_float, C.POINTER(i32), C.POINTER(C.c_float)]
        L.hp_set_workspace.argtypes = [vp, vp, C.c_size_t]
        L.hp_build_table.argtypes = [vp, vp, i64, C.POINTER(Camera), C.c_float, vp]
        L.hp_table_info.argtypes = [vp, C.POINTER(Table)]
        L.hp_table_copy.argtypes = [vp, vp, vp, vp]
        L.hp_search_sample.argtypes = [vp, vp, i64, i32, i32, C.POINTER(Samples), vp]
        L.hp_aggregate_render.argtypes = [vp, C.POINTER(Samples), i64, vp, i32, C.POINTER(Mlp), vp, vp, vp]
        L.hp_aggregate_render_backward.argtypes = [vp, C.POINTER(Samples), i64, vp, vp, i32, C.POINTER(Mlp), vp, vp,
                                                   vp, vp, vp]
        L.hp_get_status.argtypes = [vp, vp, C.POINTER(i32), C.POINTER(i64)]
        L.hp_debug_fault.argtypes = [vp, i32, i32]
        L.hp_profile_start.argtypes = [vp, i32]
        L.hp_profile_stop.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(i32), C.POINTER(i32)]
        L.hp_profile_kernel_name.argtypes = [i32]
        L.hp_profile_kernel_name.restype = C.c_char_p
        L.hp_scan_noalloc.argtypes = [vp, vp, i64, vp, vp]
        L.hp_proposal_infer.argtypes = [vp, vp, i64, vp, vp, vp]
        L.hp_proposal_train_step.argtypes = [vp, vp, i64, C.POINTER(Samples), vp, vp, vp, vp, vp, i32, C.c_float, vp,
                                             vp]
        L.hp_search_sample_proposal.argtypes = [vp, vp, i64, i32, i32, vp, C.POINTER(Samples), vp, vp]
        L.hp_search_sample_learned.argtypes = [vp, vp, i64, i32, i32, vp, C.POINTER(Samples), vp, vp]
        L.hp_selftest_mma.argtypes = [vp, vp, vp, vp, i32, i32, i32, vp]
        L.hp_status_string.argtypes = [i32]
        L.hp_status_string.restype = C.c_char_p
        L.hp_version.restype = i32
        for name in SYMBOLS:
            if name not in ("hp_status_string", "hp_version", "hp_profile_kernel_name"):
                getattr(L, name).restype = i32
        _lib = L
    return _lib


def status_string(code: int) -> str:
    return lib().hp_status_string(int(code)).decode()


def window(params, camera):
    """(h, r_ddot) of the search window (host-only call)."""
    h, rdd = C.c_int32(), C.c_float()
    _check(lib().hp_window(C.byref(config_struct(params)), C.byref(camera_struct(camera)), float(params.r),
                           C.byref(h), C.byref(rdd)), "hp_window")
    return h.value, rdd.value


def workspace_size(params, camera, n_points: int, n_rays: int, n_samples: int, K: int = None) -> int:
    n = C.c_size_t()
    K = params.K if K is None else K
    _check(lib().hp_workspace_size(C.byref(config_struct(params)), C.byref(camera_struct(camera)), float(params.r),
                                   int(n_points), int(n_rays), int(K), int(n_samples), C.byref(n)), "hp_workspace_size")
    return n.value


def scan_noalloc(d_in: torch.Tensor, d_out: torch.Tensor, d_status: Optional[torch.Tensor] = None, stream=None):
    """Exclusive prefix sum of uint32 values (int32 tensors) through the
    allocation-free entry point hp_scan_noalloc: for callers that may not
    allocate device memory; its scratch is a fixed static device array."""
    assert d_in.is_cuda and d_out.is_cuda and d_in.dtype == torch.int32 and d_out.dtype == torch.int32
    assert d_in.is_contiguous() and d_out.is_contiguous() and d_out.numel() >= d_in.numel()
    assert d_in.data_ptr() % 16 == 0 and d_out.data_ptr() % 16 == 0, \
        "hp_scan_noalloc reads and writes 16-byte vectors: both buffers must start 16-byte aligned"
    _check(lib().hp_scan_noalloc(_ptr(d_in), _ptr(d_out), d_in.numel(), _ptr(d_status), _stream(stream)),
           "hp_scan_noalloc")


def _check(rc: int, where: str):
    if rc != HP_OK:
        raise HPError(rc, where)


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream: Optional[torch.cuda.Stream]):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def camera_struct(cam) -> Camera:
    c = Camera()
    c.width, c.height = int(cam.width), int(cam.height)
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.R[:] = [float(v) for v in cam.R.reshape(-1)]
    c.t[:] = [float(v) for v in cam.t.reshape(-1)]
    c.t_near, c.t_far, c.z_near = float(cam.t_near), float(cam.t_far), float(cam.z_near)
    return c


def config_struct(p) -> Config:
    c = Config()
    c.radius_mode, c.rho = int(p.radius_mode), float(p.rho)
    c.gamma, c.beta2, c.eps_w, c.gap_k, c.eps_d = float(p.gamma), float(p.beta2), float(p.eps_w), float(p.gap_k), float(p.eps_d)
    c.cand_cap, c.bg_mode, c.window_h = int(p.cand_cap), int(p.bg_mode), int(p.window_h)
    return c


@dataclasses.dataclass
class SampleBuffers:
    """Device tensors of one hp_search_sample call (see hp_samples)."""

    n_s: torch.Tensor
    primary: torch.Tensor
    cand_count: torch.Tensor
    sample_offset: torch.Tensor
    t: torch.Tensor
    ray: torch.Tensor
    src: torch.Tensor
    delta: torch.Tensor
    nbr: Optional[torch.Tensor]          # None: the lists stay in the search's workspace
    nbr_dist: Optional[torch.Tensor]
    K: int

    @property
    def capacity(self) -> int:
        return self.t.shape[0]

    def struct(self) -> Samples:
        s = Samples()
        for f in ("n_s", "primary", "cand_count", "sample_offset", "t", "ray", "src", "delta", "nbr", "nbr_dist"):
            v = getattr(self, f)
            setattr(s, f, 0 if v is None else v.data_ptr())
        s.capacity = self.capacity
        return s

    @staticmethod
    def allocate(R: int, K: int, n_samples: int, device, capacity: Optional[int] = None,
                 lists: bool = True) -> "SampleBuffers":
        """lists=False: no packed neighbour lists (nbr, nbr_dist None); the
        search leaves them in its workspace for aggregate_render."""
        cap = R * n_samples if capacity is None else capacity
        cap1 = max(cap, 1)
        i32 = dict(dtype=torch.int32, device=device)
        f32 = dict(dtype=torch.float32, device=device)
        return SampleBuffers(
            n_s=torch.empty(max(R, 1), **i32), primary=torch.empty(max(R, 1), **i32),
            cand_count=torch.empty(max(R, 1), **i32),
            sample_offset=torch.empty(R + 1, dtype=torch.int64, device=device),
            t=torch.empty(cap1, **f32)[:cap], ray=torch.empty(cap1, **i32)[:cap], src=torch.empty(cap1, **i32)[:cap],
            delta=torch.empty(cap1, **f32)[:cap],
            nbr=torch.empty(cap1 * K, **i32)[: cap * K].view(cap, K) if lists else None,
            nbr_dist=torch.empty(cap1 * K, **f32)[: cap * K].view(cap, K) if lists else None, K=K)

    def packed(self, R: int) -> Dict[str, torch.Tensor]:
        """Host copies trimmed to the S samples written (syncs)."""
        S = int(self.sample_offset[R].item())
        S = min(S, self.capacity)
        return dict(S=S, n_s=self.n_s[:R].cpu(), primary=self.primary[:R].cpu(), cand_count=self.cand_count[:R].cpu(),
                    sample_offset=self.sample_offset.cpu(), t=self.t[:S].cpu(), ray=self.ray[:S].cpu(),
                    src=self.src[:S].cpu(), delta=self.delta[:S].cpu(),
                    nbr=None if self.nbr is None else self.nbr[:S].cpu(),
                    nbr_dist=None if self.nbr_dist is None else self.nbr_dist[:S].cpu())


class HashPoint:
    """One hot-path context (hp_ctx) on the current CUDA device."""

    def __init__(self, params, device: Optional[torch.device] = None):
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.params = params
        self._cfg = config_struct(params)
        self._ctx = C.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib().hp_create(C.byref(self._ctx), C.byref(self._cfg)), "hp_create")
        self._ws = None
        self._cam = None
        self.n_points = 0

    def close(self):
        if self._ctx:
            lib().hp_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- workspace (torch-allocated)
    def reserve(self, camera, r: float, n_points: int, n_rays: int, n_samples: int, K: int = None):
        n = C.c_size_t()
        K = self.params.K if K is None else K
        _check(lib().hp_workspace_size(C.byref(self._cfg), C.byref(camera_struct(camera)), float(r), int(n_points),
                                       int(n_rays), int(K), int(n_samples), C.byref(n)), "hp_workspace_size")
        if self._ws is None or self._ws.numel() < n.value:
            self._ws = torch.empty(n.value, dtype=torch.uint8, device=self.device)
            _check(lib().hp_set_workspace(self._ctx, _ptr(self._ws), n.value), "hp_set_workspace")
        return n.value

    # -- the three stages
    def build_table(self, points: torch.Tensor, camera, r: float, stream=None):
        assert points.is_cuda and points.dtype == torch.float32 and points.is_contiguous() and points.shape[-1] == 3
        self._cam = camera
        self.n_points = points.shape[0]
        _check(lib().hp_build_table(self._ctx, _ptr(points), points.shape[0], C.byref(camera_struct(camera)),
                                    float(r), _stream(stream)), "hp_build_table")

    def table_info(self) -> Table:
        t = Table()
        _check(lib().hp_table_info(self._ctx, C.byref(t)), "hp_table_info")
        return t

    def table(self, stream=None) -> Dict[str, torch.Tensor]:
        info = self.table_info()
        start = torch.empty(info.n_buckets + 1, dtype=torch.int32, device=self.device)
        pts = torch.empty(max(self.n_points, 1), 4, dtype=torch.float32, device=self.device)
        _check(lib().hp_table_copy(self._ctx, _ptr(start), _ptr(pts), _stream(stream)), "hp_table_copy")
        return dict(h=info.h, padded_width=info.padded_width, padded_height=info.padded_height,
                    r_ddot=info.r_ddot, start=start, points=pts[: self.n_points])

    def search_sample(self, rays: Optional[torch.Tensor], K: int, n_samples: int,
                      out: Optional[SampleBuffers] = None, stream=None) -> SampleBuffers:
        if rays is not None:
            assert rays.is_cuda and rays.dtype == torch.int32 and rays.is_contiguous()
            R = rays.shape[0]
        else:
            R = self._cam.width * self._cam.height
        if out is None:
            out = SampleBuffers.allocate(R, K, n_samples, self.device)
        s = out.struct()
        _check(lib().hp_search_sample(self._ctx, _ptr(rays), R, int(K), int(n_samples), C.byref(s), _stream(stream)),
               "hp_search_sample")
        self._R = R
        return out

    def search_sample_proposal(self, rays: Optional[torch.Tensor], K: int, n_samples: int, interval: torch.Tensor,
                               out: Optional[SampleBuffers] = None, fallback_count: Optional[torch.Tensor] = None,
                               stream=None) -> SampleBuffers:
        """search_sample restricted to per-ray intervals with the plain search as
        fallback; fallback_count (int32[1] device, optional) gets the number of
        rays searched again."""
        R = rays.shape[0] if rays is not None else self._cam.width * self._cam.height
        if out is None:
            out = SampleBuffers.allocate(R, K, n_samples, self.device)
        s = out.struct()
        _check(lib().hp_search_sample_proposal(self._ctx, _ptr(rays), R, int(K), int(n_samples), _ptr(interval),
                                               C.byref(s), _ptr(fallback_count), _stream(stream)),
               "hp_search_sample_proposal")
        self._R = R
        return out

    def search_sample_learned(self, rays: Optional[torch.Tensor], K: int, n_samples: int, weights_bf16: torch.Tensor,
                              out: Optional[SampleBuffers] = None, fallback_count: Optional[torch.Tensor] = None,
                              stream=None) -> SampleBuffers:
        """search_sample_proposal with the intervals inferred inside the search
        from the BF16 proposal weights (same results as proposal_infer followed
        by search_sample_proposal)."""
        assert weights_bf16.is_cuda and weights_bf16.numel() == PROP_PARAMS
        R = rays.shape[0] if rays is not None else self._cam.width * self._cam.height
        if out is None:
            out = SampleBuffers.allocate(R, K, n_samples, self.device)
        s = out.struct()
        _check(lib().hp_search_sample_learned(self._ctx, _ptr(rays), R, int(K), int(n_samples), _ptr(weights_bf16),
                                              C.byref(s), _ptr(fallback_count), _stream(stream)),
               "hp_search_sample_learned")
        self._R = R
        return out

    def proposal_infer(self, rays: Optional[torch.Tensor], weights_bf16: torch.Tensor,
                       interval: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        R = rays.shape[0] if rays is not None else self._cam.width * self._cam.height
        if interval is None:
            interval = torch.empty(max(R, 1), 2, dtype=torch.float32, device=self.device)[:R]
        _check(lib().hp_proposal_infer(self._ctx, _ptr(rays), R, _ptr(weights_bf16), _ptr(interval),
                                       _stream(stream)), "hp_proposal_infer")
        return interval

    def proposal_train_step(self, rays: Optional[torch.Tensor], plain: SampleBuffers, state: "ProposalState",
                            lr: float = 3e-3, stream=None) -> None:
        R = rays.shape[0] if rays is not None else self._cam.width * self._cam.height
        state.step += 1
        s = plain.struct()
        _check(lib().hp_proposal_train_step(self._ctx, _ptr(rays), R, C.byref(s), _ptr(state.params), _ptr(state.m),
                                            _ptr(state.v), _ptr(state.grad), _ptr(state.bf16), state.step, float(lr),
                                            _ptr(state.loss), _stream(stream)), "hp_proposal_train_step")

    def aggregate_render(self, samples: SampleBuffers, feats: torch.Tensor, mlp_dims: Sequence[int],
                         mlp_params: torch.Tensor, rgb: Optional[torch.Tensor] = None,
                         wsum: Optional[torch.Tensor] = None, stream=None, decode: int = DECODE_FP32):
        assert feats.is_cuda and feats.dtype == torch.float32 and feats.is_contiguous()
        assert mlp_params.is_cuda and mlp_params.dtype == torch.float32 and mlp_params.is_contiguous()
        R = self._R
        if rgb is None:
            rgb = torch.empty(max(R, 1), 3, dtype=torch.float32, device=self.device)[:R]
        if wsum is None:
            wsum = torch.empty(max(R, 1), dtype=torch.float32, device=self.device)[:R]
        m = Mlp()
        m.n_layers = len(mlp_dims) - 1
        for i, d in enumerate(mlp_dims):
            m.dims[i] = int(d)
        m.d_params = mlp_params.data_ptr()
        m.decode = int(decode)
        s = samples.struct()
        _check(lib().hp_aggregate_render(self._ctx, C.byref(s), R, _ptr(feats), feats.shape[1], C.byref(m),
                                         _ptr(rgb), _ptr(wsum), _stream(stream)), "hp_aggregate_render")
        return rgb, wsum

    def render(self, points, feats, camera, mlp_dims, mlp_params, rays=None, stream=None, samples=None,
               decode: int = DECODE_FP32):
        """build_table + search_sample + aggregate_render for one frame."""
        p = self.params
        self.build_table(points, camera, p.r, stream)
        smp = self.search_sample(rays, p.K, p.n_max, out=samples, stream=stream)
        rgb, wsum = self.aggregate_render(smp, feats, mlp_dims, mlp_params, stream=stream, decode=decode)
        return rgb, wsum, smp

    def aggregate_render_backward(self, samples: SampleBuffers, points: torch.Tensor, feats: torch.Tensor,
                                  mlp_dims: Sequence[int], mlp_params: torch.Tensor, grad_rgb: torch.Tensor,
                                  grad_wsum: Optional[torch.Tensor] = None, grad_feats: Optional[torch.Tensor] = None,
                                  grad_points: Optional[torch.Tensor] = None, stream=None, want_points: bool = True):
        """Accumulate dL/dfeats (N x F) and dL/dpoints (N x 3, world) for the
        output gradients of the last aggregate_render (structure frozen).
        want_points=False skips the position gradient (returns None for it)."""
        R = self._R
        N, F = feats.shape
        grad_rgb = grad_rgb.contiguous().float()
        assert grad_rgb.numel() == 3 * R and points.shape == (N, 3)
        if grad_wsum is not None:
            grad_wsum = grad_wsum.contiguous().float()
            assert grad_wsum.numel() == R
        if grad_feats is None:
            grad_feats = torch.zeros_like(feats)
        assert grad_feats.is_contiguous() and grad_feats.dtype == torch.float32 and grad_feats.numel() == N * F
        if not want_points:
            grad_points = None
        elif grad_points is None:
            grad_points = torch.zeros_like(points)
        if grad_points is not None:
            assert grad_points.is_contiguous() and grad_points.dtype == torch.float32 and grad_points.numel() == 3 * N
        m = Mlp()
        m.n_layers = len(mlp_dims) - 1
        for i, d in enumerate(mlp_dims):
            m.dims[i] = int(d)
        m.d_params = mlp_params.data_ptr()
        s = samples.struct()
        _check(lib().hp_aggregate_render_backward(self._ctx, C.byref(s), R, _ptr(points), _ptr(feats), feats.shape[1],
                                                  C.byref(m), _ptr(grad_rgb), _ptr(grad_wsum), _ptr(grad_feats),
                                                  _ptr(grad_points), _stream(stream)), "hp_aggregate_render_backward")
        return grad_feats, grad_points

    def selftest_mma(self, A: torch.Tensor, B: torch.Tensor, bf16: bool = False, a_tmem: bool = False,
                     stream=None) -> torch.Tensor:
        """D = A B^T on the tensor cores (A 128 x K, B N x K, fp16 or bf16;
        a_tmem: A read from tensor memory)."""
        assert A.shape[0] == 128 and A.shape[1] == B.shape[1] and A.is_contiguous() and B.is_contiguous()
        D = torch.empty(128, B.shape[0], dtype=torch.float32, device=A.device)
        flags = (1 if bf16 else 0) | (2 if a_tmem else 0)
        _check(lib().hp_selftest_mma(self._ctx, _ptr(A), _ptr(B), _ptr(D), A.shape[1], B.shape[0], flags,
                                     _stream(stream)), "hp_selftest_mma")
        return D

    def status(self, stream=None):
        code, detail = C.c_int32(), C.c_int64()
        _check(lib().hp_get_status(self._ctx, _stream(stream), C.byref(code), C.byref(detail)), "hp_get_status")
        return code.value, detail.value

    def profile_start(self, max_launches: int = 4096):
        _check(lib().hp_profile_start(self._ctx, int(max_launches)), "hp_profile_start")

    def profile_stop(self):
        """{kernel name: (total ms, timed launches, CUDA kernels run)} since
        profile_start (syncs)."""
        ms = (C.c_double * PROF_KERNELS)()
        n = (C.c_int32 * PROF_KERNELS)()
        nk = (C.c_int32 * PROF_KERNELS)()
        _check(lib().hp_profile_stop(self._ctx, ms, n, nk), "hp_profile_stop")
        return {lib().hp_profile_kernel_name(i).decode(): (ms[i], n[i], nk[i]) for i in range(PROF_KERNELS)}

    def debug_fault(self, skip_tile: int, spin_limit: int = 0):
        _check(lib().hp_debug_fault(self._ctx, int(skip_tile), int(spin_limit)), "hp_debug_fault")


class ProposalState:
    """FP32 master weights, Adam moments, gradient, BF16 copy and loss of the
    proposal MLP (device tensors)."""

    def __init__(self, device, seed: int = 0, init: Optional[torch.Tensor] = None):
        if init is not None:
            self._set(device, init.detach().float().reshape(-1))
            return
        g = torch.Generator().manual_seed(seed)
        shapes = [(32, PROP_BINS), (32,), (32, 32), (32,), (2, 32), (2,)]
        parts = []
        for sh in shapes:
            if len(sh) == 2:
                lim = (6.0 / sh[1]) ** 0.5
                parts.append((torch.rand(sh, generator=g) * 2 - 1).mul(lim).reshape(-1))
            else:
                parts.append(torch.zeros(sh))
        # start wide: t0 near t_near, t1 near t_far
        parts[-1] = torch.tensor([-3.0, 3.0])
        self._set(device, torch.cat(parts))

    def _set(self, device, params):
        self.params = params.to(device).contiguous()
        assert self.params.numel() == PROP_PARAMS
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad = torch.zeros_like(self.params)
        self.refresh_bf16()
        self.loss = torch.zeros(2, device=device)
        self.step = 0

    def refresh_bf16(self):
        """The inference copy: the FP32 weights rounded to bfloat16 (nearest even)."""
        self.bf16 = self.params.to(torch.bfloat16).view(torch.int16).contiguous()

    # Checkpoint file: 8-byte magic, little-endian uint64 header length, a JSON
    # header, then the FP32 arrays it lists (parameters, Adam's m and v), raw
    # little-endian, in that order.  Enough to resume training (Adam's step
    # count is in the header) or to serve the network (its BF16 copy is
    # re-derived from the parameters on load).
    MAGIC = b"HPPROP\x00\x01"

    def save(self, path: str) -> None:
        header = {"format": "hashpoint-proposal", "version": 1, "layers": [PROP_BINS, 32, 32, 2],
                  "n_params": PROP_PARAMS, "dtype": "float32", "byteorder": "little", "step": int(self.step),
                  "arrays": ["params", "m", "v"]}
        raw = json.dumps(header, sort_keys=True).encode()
        tmp = path + ".tmp"
        with open(tmp, "wb") as f:
            f.write(self.MAGIC)
            f.write(struct.pack("<Q", len(raw)))
            f.write(raw)
            for t in (self.params, self.m, self.v):
                f.write(t.detach().to("cpu", torch.float32).contiguous().numpy().astype("<f4").tobytes())
        os.replace(tmp, path)

    @classmethod
    def load(cls, path: str, device) -> "ProposalState":
        with open(path, "rb") as f:
            blob = f.read()
        if blob[:8] != cls.MAGIC or len(blob) < 16:
            raise ValueError(f"{path}: not a proposal checkpoint")
        (n,) = struct.unpack("<Q", blob[8:16])
        header = json.loads(blob[16:16 + n].decode())
        if header.get("format") != "hashpoint-proposal" or header.get("version") != 1 or \
                header.get("n_params") != PROP_PARAMS or header.get("dtype") != "float32":
            raise ValueError(f"{path}: unsupported proposal checkpoint header {header}")
        body = blob[16 + n:]
        if len(body) != 3 * 4 * PROP_PARAMS:
            raise ValueError(f"{path}: expected {3 * 4 * PROP_PARAMS} bytes of arrays, found {len(body)}")
        import numpy as np
        arr = np.frombuffer(body, dtype="<f4").reshape(3, PROP_PARAMS)
        st = cls.__new__(cls)
        st._set(device, torch.from_numpy(arr[0].copy()))
        st.m = torch.from_numpy(arr[1].copy()).to(device).contiguous()
        st.v = torch.from_numpy(arr[2].copy()).to(device).contiguous()
        st.step = int(header["step"])
        return st


class RenderFunction(torch.autograd.Function):
    """Differentiable frame: (feats, points) -> (rgb, wsum) through the
    library's forward kernels and its backward kernels.  The search and
    selection are treated as constants (index outputs)."""

    @staticmethod
    def forward(ctx, feats, points, hp, camera, mlp_dims, mlp_params, rays, decode):
        rgb, wsum, smp = hp.render(points.detach().contiguous(), feats.detach().contiguous(), camera, mlp_dims,
                                   mlp_params, rays=rays, decode=decode)
        ctx.hp, ctx.smp, ctx.mlp_dims, ctx.mlp_params = hp, smp, list(mlp_dims), mlp_params
        ctx.save_for_backward(feats, points)
        return rgb, wsum

    @staticmethod
    def backward(ctx, grad_rgb, grad_wsum):
        feats, points = ctx.saved_tensors
        if grad_rgb is None:
            grad_rgb = torch.zeros(ctx.hp._R, 3, device=feats.device)
        gf, gp = ctx.hp.aggregate_render_backward(ctx.smp, points.detach().contiguous(), feats.detach().contiguous(),
                                                  ctx.mlp_dims, ctx.mlp_params, grad_rgb, grad_wsum)
        return gf, gp, None, None, None, None, None, None


def render_differentiable(hp: HashPoint, feats, points, camera, mlp_dims, mlp_params, rays=None, decode=DECODE_FP32):
    """rgb (R x 3), wsum (R) with autograd to feats and points."""
    return RenderFunction.apply(feats, points, hp, camera, mlp_dims, mlp_params, rays, decode)
