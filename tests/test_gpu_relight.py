"""Tensor-core relighting under many environment lights (avatar_shade_multi).

D = vis*cos and S = D*f_s enter the tensor cores as BF16 (relative rounding
2^-9 per term) with FP32 accumulation; the stated bound for this form is a
max-abs colour error of 1e-3 against both the FP64 oracle and the FP32
single-light path on the same inputs.
"""
import numpy as np
import pytest

from _common import O, f32, light_ordered_bits, oracle_frame, scene

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TC_TOL = 1e-3


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    from paper_2407_10707_gb300 import api
    return api


def T(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _inputs(name, n_env, seed):
    sc = scene(name)
    ref = oracle_frame(name)
    sk = ref["skin"]
    ins = {k: f32(sk[k]) for k in ("xd", "nd", "ag", "rg", "pg", "ubar")}
    rng = np.random.default_rng(seed)
    env = np.exp(rng.normal(-1.0, 0.5, size=(n_env,) + sc.light.L.shape)).astype(np.float32)
    return sc, ref, ins, env


@pytest.mark.parametrize("name,n_env", [("c1_small", 5), ("c1_small", 32), ("c3_fd", 1)])
def test_multi_light_matches_oracle_and_fp32_path(gpu, name, n_env):
    api = gpu
    sc, ref, ins, env = _inputs(name, n_env, seed=n_env)
    cam_c = f32(sc.camera.center)
    A, w = f32(sc.light.A), f32(sc.light.w)
    bits_l = light_ordered_bits(ref["bits"], sc.dmap)
    skt = {k: T(v.T if v.ndim == 2 else v) for k, v in ins.items()}
    knn = T(sc.avatar.knn.T, torch.int32)
    bits = T(bits_l.view(np.int32), torch.int32)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    cull = torch.full((sc.avatar.G,), 7, dtype=torch.uint8, device="cuda")
    out = torch.full((n_env, 3, sc.avatar.G), float("nan"), device="cuda")
    api.avatar_shade_multi(skt, knn, bits, dict(A=T(A), w=T(w)), cam_c, T(env), out=out, cull=cull, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    got = out.cpu().numpy()
    assert np.isfinite(got).all()   # every colour written: live by the tiles, culled by the first pass
    mcull = cull.cpu().numpy()
    worst_oracle = worst_fp32 = 0.0
    for l in range(n_env):
        col_ref, _, cull_ref = O.shade(*(ins[k].astype(np.float64) for k in ("xd", "nd", "ag", "rg", "pg", "ubar")),
                                       sc.avatar.knn, ref["bits"], env[l].astype(np.float64), A.astype(np.float64),
                                       w.astype(np.float64), sc.dmap, cam_c.astype(np.float64), sc.frames.shape[0])
        one = api.avatar_shade(skt, knn, bits, dict(L=T(env[l]), A=T(A), w=T(w)), cam_c)
        torch.cuda.synchronize()
        fp32 = one["color"].cpu().numpy()
        assert np.array_equal(one["cull"].cpu().numpy(), cull_ref)
        assert np.array_equal(mcull, cull_ref)
        g = got[l]
        assert np.all(g[:, cull_ref == 1] == 0)
        worst_oracle = max(worst_oracle, float(np.abs(g.T - col_ref).max()))
        worst_fp32 = max(worst_fp32, float(np.abs(g - fp32).max()))
    print(f"{name} n_env={n_env}: max|tc - fp64| {worst_oracle:.2e}, max|tc - fp32| {worst_fp32:.2e}")
    assert worst_oracle < TC_TOL
    assert worst_fp32 < TC_TOL


def test_multi_light_rejects_unsupported_sizes(gpu):
    api = gpu
    sc, ref, ins, env = _inputs("c3_fd", 1, seed=0)
    skt = {k: T(v.T if v.ndim == 2 else v) for k, v in ins.items()}
    knn = T(sc.avatar.knn.T, torch.int32)
    bits = T(light_ordered_bits(ref["bits"], sc.dmap).view(np.int32), torch.int32)
    light = dict(A=T(f32(sc.light.A)), w=T(f32(sc.light.w)))
    with pytest.raises(Exception):   # more than 32 lights at once
        api.avatar_shade_multi(skt, knn, bits, light, f32(sc.camera.center), T(np.ones((33, 128, 3), np.float32)))


def test_multi_light_workspace_and_index_errors(gpu):
    api = gpu
    from paper_2407_10707_gb300 import _lib as L
    sc, ref, ins, env = _inputs("c3_fd", 2, seed=1)
    skt = {k: T(v.T if v.ndim == 2 else v) for k, v in ins.items()}
    knn_np = sc.avatar.knn.T.copy()
    bits = T(light_ordered_bits(ref["bits"], sc.dmap).view(np.int32), torch.int32)
    light = dict(A=T(f32(sc.light.A)), w=T(f32(sc.light.w)))
    with pytest.raises(L.AvatarError):   # a workspace one byte short
        _short_ws(api, skt, T(knn_np, torch.int32), bits, light, f32(sc.camera.center), T(env))
    bad = knn_np.copy()
    bad[1, 5] = sc.avatar.Nv            # one neighbour index out of range
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    cull = torch.zeros(sc.avatar.G, dtype=torch.uint8, device="cuda")
    out = api.avatar_shade_multi(skt, T(bad, torch.int32), bits, light, f32(sc.camera.center), T(env),
                                 cull=cull, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 7      # AVATAR_ERR_INDEX
    assert int(cull[5].item()) == 1 and float(out[:, :, 5].abs().max()) == 0.0


def _short_ws(api, skt, knn, bits, light, cam, env):
    import ctypes as C
    from paper_2407_10707_gb300 import _lib as L
    lib = L.load()
    m = L.ShadeMultiArgs()
    G = skt["xd"].shape[1]
    out = torch.empty(env.shape[0], 3, G, device="cuda")
    m.base = api._shade_struct(skt, knn, bits, dict(light, L=env[0]), cam, None, None, None, None)
    m.n_env, m.env_L, m.env_color = env.shape[0], env.data_ptr(), out.data_ptr()
    need = lib.avatar_shade_multi_workspace_size(C.byref(m))
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    m.workspace, m.workspace_bytes = ws.data_ptr(), need - 1
    L.check(lib.avatar_shade_multi(api.context(), C.byref(m), None), "avatar_shade_multi")
