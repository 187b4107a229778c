"""The C-ABI library builds for sm_103a, loads, and exports every entry
point include/avatar.h declares (no compute call: runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "avatar.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w\s\*]+?\b(avatar_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    import __graft_entry__ as ge
    ge.build()
    from paper_2407_10707_gb300 import _lib
    lib = ctypes.CDLL(_lib.LIB_PATH)
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the Python binding covers the same set
    assert set(names) == set(_lib.EXPORTED), set(names) ^ set(_lib.EXPORTED)


def test_host_only_calls_without_a_gpu():
    from paper_2407_10707_gb300 import _lib
    lib = _lib.load()
    assert lib.avatar_status_string(3) == b"tile/Gaussian pair buffer overflow"
    assert lib.avatar_version() >= 10000
    # argument validation happens on the host, before any CUDA call
    a = _lib.SplatArgs()
    a.G = 10
    a.cam.width = a.cam.height = 64
    a.tile = 12
    assert lib.avatar_splat_num_tiles(ctypes.byref(a)) == 0
    a.tile = 16
    assert lib.avatar_splat_workspace_size(ctypes.byref(a)) == 0   # pair_capacity missing
    v = _lib.VisArgs()
    v.Nv, v.F, v.D, v.R = 100, 10, 30, 64
    assert lib.avatar_visibility_workspace_size(ctypes.byref(v)) == 0   # D not a multiple of 32


def test_product_path_refuses_to_run_without_cuda(monkeypatch):
    import pytest
    import torch
    from paper_2407_10707_gb300 import api
    monkeypatch.setattr(torch.cuda, "is_available", lambda: False)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        api.context()
