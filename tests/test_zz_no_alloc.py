"""The allocation-free prefix sum (hp_scan_noalloc) against the table build.

Some callers cannot let a library allocate device memory -- an application
that owns the whole memory budget, or a real-time loop where a cudaMalloc
would stall -- so hp_scan_noalloc keeps its scratch in a fixed static device
array.  Its result must equal the bucket starts that the regular entry point
hp_build_table computes with its own workspace.  Two calls run back to back
(different sizes) so that contents the shared array keeps from a previous
call cannot leak into the next one.  This file is collected last."""
import numpy as np
import pytest
import torch

from paper_2404_14044_b300 import scenes

pytestmark = pytest.mark.gpu


def _table_starts(hp, pts, cam, r):
    hp.build_table(pts, cam, r)
    tb = hp.table()
    assert hp.status() == (0, 0)
    return tb["start"]                     # int32 view of the uint32 starts, n_buckets + 1


def test_scan_noalloc_matches_build_table_twice():
    from paper_2404_14044_b300 import hashpoint as H
    dev = torch.device("cuda", 0)
    pts_np = scenes.object_points(300_000, 0)
    pts = torch.from_numpy(pts_np).to(dev)
    params = scenes.Params(r=0.005, K=8, n_max=8)
    hp = H.HashPoint(params, dev)
    status = torch.full((1,), -1, dtype=torch.int32, device=dev)
    sizes = []
    for res, view in ((800, 0), (333, 1)):                 # a large then a smaller, ragged call
        cam = scenes.random_sphere_cameras(view + 1, 4.0, 0, width=res, height=res)[view]
        start = _table_starts(hp, pts, cam, params.r)
        counts = torch.zeros_like(start)
        counts[:-1] = start[1:] - start[:-1]               # per-bucket counts, last entry 0
        out = torch.full_like(start, -7)
        H.scan_noalloc(counts, out, status)
        torch.cuda.synchronize()
        assert int(status.item()) == H.HP_OK
        assert torch.equal(out, start)                     # integers: exact
        sizes.append(start.numel())
    assert sizes[0] > sizes[1]
    hp.close()


def test_scan_noalloc_rejects_too_large():
    from paper_2404_14044_b300 import hashpoint as H
    dev = torch.device("cuda", 0)
    x = torch.zeros(16, dtype=torch.int32, device=dev)
    rc = H.lib().hp_scan_noalloc(H._ptr(x), H._ptr(x), H.SCAN_NOALLOC_MAX_N + 1, None, H._stream(None))
    assert rc == H.HP_ERR_TOO_LARGE


def _wrapping_exclusive_scan(x: np.ndarray) -> np.ndarray:
    inc = np.cumsum(x.astype(np.uint64)) & np.uint64(0xFFFFFFFF)
    out = np.zeros_like(x, dtype=np.uint32)
    out[1:] = inc[:-1].astype(np.uint32)
    return out


@pytest.mark.parametrize("kind", ["all_ones", "near_2_31", "full_range"])
def test_scan_noalloc_wrapping_uint32(kind):
    """Sums past 2^31 and 2^32 inside and across the scan's 8192-entry tiles,
    on a ragged length: the result must equal the uint32 exclusive prefix sum
    modulo 2^32."""
    from paper_2404_14044_b300 import hashpoint as H
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(7)
    n = 5 * 8192 + 777
    if kind == "all_ones":
        x = np.full(n, 0xFFFFFFFF, dtype=np.uint32)
    elif kind == "near_2_31":
        x = (np.uint32(1 << 31) - rng.integers(0, 1000, n).astype(np.uint32)).astype(np.uint32)
    else:
        x = rng.integers(0, 1 << 32, n, dtype=np.uint64).astype(np.uint32)
    d_in = torch.from_numpy(x.view(np.int32).copy()).to(dev)
    status = torch.full((1,), -1, dtype=torch.int32, device=dev)
    for _ in range(2):                                    # the shared array is reused by the second call
        d_out = torch.full((n,), -7, dtype=torch.int32, device=dev)
        H.scan_noalloc(d_in, d_out, status)
        torch.cuda.synchronize()
        assert int(status.item()) == H.HP_OK
        got = d_out.cpu().numpy().view(np.uint32)
        assert np.array_equal(got, _wrapping_exclusive_scan(x))
