"""The C-ABI library without a GPU: it loads, exports every symbol the
header declares, and its host-only calls (window bound, workspace size,
argument checks) agree with the oracle and reject bad input."""
import ctypes as C
import glob
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
from paper_2404_14044_b300 import hashpoint as H
from paper_2404_14044_b300 import scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(hp_\w+)\s*\(", txt, flags=re.M))
    return names


def test_library_exports_every_declared_symbol():
    L = H.lib()
    names = declared_symbols()
    assert names == set(H.SYMBOLS), names ^ set(H.SYMBOLS)
    out = subprocess.run(["nm", "-D", "--defined-only", H.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\b(hp_\w+)$", out, flags=re.M))
    assert names <= exported
    for n in names:
        assert hasattr(L, n)
    assert L.hp_version() >= 10000


def test_status_strings():
    assert H.status_string(0) == "ok"
    assert "timed out" in H.status_string(H.HP_ERR_TIMEOUT)
    assert H.status_string(99) == "unknown status"


def _cases():
    out = []
    for name in ("sphere_plane_64",):
        sc = scenes.WORKLOADS[name]()
        out.append((sc.camera, sc.params))
    cam2 = scenes.random_sphere_cameras(3, 4.0, 0)
    for c in cam2:
        out.append((c, scenes.Params(r=0.005)))
    f = 0.8 * 1008
    fwd = scenes.Camera(1008, 756, f, f, 504.0, 378.0, np.eye(3, dtype=np.float32), np.zeros(3, np.float32), 0.5, 10.0, 0.05)
    for mode in (1, 2):
        for rho in (1.0, 2.0, 3.5, 0.0):
            out.append((fwd, scenes.Params(radius_mode=mode, rho=rho, r=0.004)))
    out.append((cam2[0], scenes.Params(r=0.01, window_h=7)))
    return out


@pytest.mark.parametrize("case", range(len(_cases())))
def test_window_matches_oracle(case):
    cam, p = _cases()[case]
    assert H.window(p, cam) == oracle.window(cam, p)


def test_workspace_size_and_bad_arguments():
    sc = scenes.sphere_plane_64()
    a = H.workspace_size(sc.params, sc.camera, 1000, 4096, 4)
    b = H.workspace_size(sc.params, sc.camera, 100000, 4096, 4)
    assert a % 256 == 0 and b > a
    bad = scenes.Params(**{**sc.params.__dict__, "gamma": 0.0})
    with pytest.raises(H.HPError) as e:
        H.window(bad, sc.camera)
    assert e.value.code == H.HP_ERR_INVALID_ARG
    for field, val in (("cand_cap", 0), ("cand_cap", 129), ("beta2", -1.0), ("radius_mode", 5), ("eps_d", 0.0)):
        with pytest.raises(H.HPError):
            H.window(scenes.Params(**{**sc.params.__dict__, field: val}), sc.camera)
    cam = scenes.Camera(**{**sc.camera.__dict__, "t_near": 0.0})
    with pytest.raises(H.HPError):
        H.window(sc.params, cam)
    with pytest.raises(H.HPError):                      # radius too large for the window limit
        H.window(scenes.Params(r=5.0), sc.camera)
    with pytest.raises(H.HPError):
        H.workspace_size(sc.params, sc.camera, 10, 10, 0)


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(H, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(H, "_lib", None)
    with pytest.raises(RuntimeError):
        H.lib()
