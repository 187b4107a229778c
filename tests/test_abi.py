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


def test_workspace_queries_validate_on_the_host():
    """Size queries need no GPU: invalid arguments give 0, valid ones a size
    that grows with the problem (pointers are never dereferenced on the host,
    so dummy non-null values stand in for device buffers)."""
    from paper_2407_10707_gb300 import _lib
    lib = _lib.load()
    dummy = ctypes.c_void_p(4096)

    def vis(**kw):
        v = _lib.VisArgs()
        v.Nv, v.F, v.D, v.R = 50_000, 100_000, 512, 256
        v.xp = v.faces = v.frames = v.bits = dummy
        for k, x in kw.items():
            setattr(v, k, x)
        return lib.avatar_visibility_workspace_size(ctypes.byref(v))

    base = vis()
    assert base > 0
    for bad in (dict(R=260), dict(R=1024), dict(D=4128), dict(D=0), dict(Nv=0), dict(bits=None)):
        assert vis(**bad) == 0, bad
    # per face: at least the packed chunk-relative word the raster reads
    assert vis(F=200_000) - base >= 100_000 * 4
    # per vertex and direction: at least one bit
    assert vis(D=1024) - base >= 50_000 * 512 // 8

    la = _lib.ImageLossArgs()
    la.C, la.H, la.W, la.lam, la.weight = 3, 1024, 1024, 0.2, 1.0
    n = lib.avatar_image_loss_workspace_size(ctypes.byref(la))
    assert n >= 3 * 3 * 1024 * 1024 * 4          # the three dSSIM coefficient maps
    for k, x in (("lam", 1.5), ("weight", -1.0), ("H", 0)):
        bad = _lib.ImageLossArgs.from_buffer_copy(la)
        setattr(bad, k, x)
        assert lib.avatar_image_loss_workspace_size(ctypes.byref(bad)) == 0, k

    a = _lib.SplatArgs()
    a.G, a.tile, a.pair_capacity = 200_000, 16, 1 << 22
    a.cam.width, a.cam.height = 1024, 1024
    assert lib.avatar_splat_num_tiles(ctypes.byref(a)) == 64 * 64
    s16 = lib.avatar_splat_workspace_size(ctypes.byref(a))
    assert s16 > 0
    a.pair_capacity = 1 << 23
    assert lib.avatar_splat_workspace_size(ctypes.byref(a)) > s16      # pair buffers scale with capacity


def test_product_path_refuses_to_run_without_cuda(monkeypatch):
    import pytest
    import torch
    from paper_2407_10707_gb300 import api
    monkeypatch.setattr(torch.cuda, "is_available", lambda: False)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        api.context()


def test_static_scratch_holds_the_paper_scale_visibility():
    """The scratch-free visibility entry point's fixed array holds the
    workspace of the paper-scale frame (50k vertices, 99,856 faces, 512
    directions at 256^2, 512 lights) and refuses the stress frame's."""
    import ctypes as C
    from paper_2407_10707_gb300 import _lib as L
    lib = L.load()
    cap = lib.avatar_visibility_static_scratch_bytes()
    for (nv, F, D, R, NL), fits in (((50_000, 99_856, 512, 256, 512), True),
                                    ((200_000, 400_000, 1024, 512, 2048), False)):
        a = L.VisArgs()
        a.Nv, a.F, a.D, a.R, a.NL = nv, F, D, R, NL
        a.xp = a.faces = a.frames = a.bits = a.dmap = C.c_void_p(256)
        a.half_extent = 1.0
        need = lib.avatar_visibility_workspace_size(C.byref(a))
        assert need > 0 and (need <= cap) == fits, (need, cap)
