"""The workspace-free visibility entry point, through the C ABI.

avatar_visibility_static_scratch serves callers that cannot allocate device
memory (a host application that owns every device allocation, or a real-time
loop where cudaMalloc is not allowed): it runs on a fixed scratch array built
into the library.  This file is collected last on purpose, so that a run
stopping at the first failure has already run every other test.  It passes
alone in a fresh process and after the other tests.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    from paper_2407_10707_gb300 import _lib as L
    from paper_2407_10707_gb300 import api, synth
    return L, api, synth


def _case(api, synth, seed, n_dirs=128, res=256, nv=4000):
    sc = synth.make_scene(nv, 10, 8, 16, n_dirs, res, 64, 64, seed)
    from oracle import oracle as O
    sk = O.skin(sc.avatar, O.fk(sc.avatar.parents, sc.avatar.joints, sc.avatar.pose))
    dev = "cuda"
    xp = torch.as_tensor(np.asarray(sk["xp"], np.float32).T.copy(), device=dev)
    faces = torch.as_tensor(sc.avatar.faces, dtype=torch.int32, device=dev)
    frames = torch.as_tensor(sc.frames.reshape(-1, 9).astype(np.float32), device=dev)
    dmap = torch.as_tensor(sc.dmap, dtype=torch.int32, device=dev)
    return sc, xp, faces, frames, dmap


def _args(api, sc, xp, faces, frames, dmap, bits, status):
    return api._vis_struct(xp, faces, frames, sc.window_center, sc.window_half, sc.vis_bias, sc.depth_res, dmap,
                           bits, status)


def test_static_scratch_matches_workspace_entry_point_on_two_calls():
    L, api, synth = _setup()
    lib = L.load()
    ctx = api.context()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.avatar_visibility_static_scratch_bytes() == 8 << 20
    # calls in a row with different inputs, a larger one (20k vertices, 512
    # directions: 1.7 MiB of scratch) before a smaller one that leaves the
    # larger call's data beyond its own layout; each must equal the
    # workspace entry point bit for bit
    for seed, nd, nv in ((11, 512, 20_000), (12, 128, 4000), (13, 128, 4000)):
        sc, xp, faces, frames, dmap = _case(api, synth, seed, n_dirs=nd, nv=nv)
        nw = (dmap.shape[0] + 31) // 32
        ref_bits = torch.full((xp.shape[1], nw), -1, dtype=torch.int32, device="cuda")
        got_bits = torch.full_like(ref_bits, 7)
        status = torch.zeros(1, dtype=torch.int32, device="cuda")
        a_ref = _args(api, sc, xp, faces, frames, dmap, ref_bits, status)
        ws = api.workspace(lib.avatar_visibility_workspace_size(C.byref(a_ref)), "cuda")
        L.check(lib.avatar_visibility(ctx, C.byref(a_ref), C.c_void_p(ws.data_ptr()), ws.numel(), stream),
                "avatar_visibility")
        a = _args(api, sc, xp, faces, frames, dmap, got_bits, status)
        L.check(lib.avatar_visibility_static_scratch(ctx, C.byref(a), stream), "avatar_visibility_static_scratch")
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        assert torch.equal(got_bits, ref_bits), f"seed {seed}: {int((got_bits != ref_bits).sum())} words differ"


def test_static_scratch_rejects_sizes_beyond_its_array():
    L, api, synth = _setup()
    lib = L.load()
    ctx = api.context()
    a = L.VisArgs()
    a.Nv, a.F, a.D, a.R = 200_000, 400_000, 1024, 256   # ~29 MB of scratch: more than 8 MiB
    a.xp = a.faces = a.frames = a.bits = C.c_void_p(16)
    a.half_extent = 1.0
    rc = lib.avatar_visibility_static_scratch(ctx, C.byref(a), None)
    assert rc == 2   # AVATAR_ERR_WORKSPACE, before any launch
