"""The paper's own visibility on the GPU (avatar_visibility_soft): triangle-ID
images and the median / median / mean vertex filters (Sec. 3.2, Eqs. 3-4).

Every step is integer, so the unfiltered visibility V and the filtered counts
Kv * Vbar must equal the FP64/integer oracle bit for bit given the same FP32
posed vertices.  Soft-visibility shading is FP32 against the FP64 oracle
(5e-5 of the largest radiance, as for the bit form); with counts of 0 or Kv it
reduces to the bit form.
"""
import numpy as np
import pytest

from _common import O, f32, light_ordered_bits, oracle_frame, rel_err, scene, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KV = 19


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


def _inputs(name):
    sc = scene(name)
    av = sc.avatar
    sk = O.skin(av, O.fk(av.parents, av.joints, av.pose))
    xp = f32(sk["xp"])
    knn_v = synth.vertex_knn(av.xv, KV)
    return sc, xp, knn_v


@pytest.mark.parametrize("name,cull_back", [("c1_small", False), ("c1_small", True), ("c3_fd", False)])
def test_raw_and_filtered_visibility_bit_exact(gpu, name, cull_back):
    api = gpu
    sc, xp, knn_v = _inputs(name)
    av = sc.avatar
    D = sc.frames.shape[0]
    fr = f32(sc.frames.reshape(-1, 9))
    raw = torch.empty(av.Nv, D // 32, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    cnt = api.avatar_visibility_soft(T(xp.T), T(av.faces, torch.int32), T(fr), sc.window_center, sc.window_half,
                                     sc.depth_res, T(knn_v.T, torch.int32), raw_bits=raw, status=status,
                                     cull_back=cull_back)
    cnt_l = api.avatar_visibility_soft(T(xp.T), T(av.faces, torch.int32), T(fr), sc.window_center,
                                       sc.window_half, sc.depth_res, T(knn_v.T, torch.int32),
                                       dmap=T(sc.dmap, torch.int32), status=status, cull_back=cull_back)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    # the window reaches the library as FP32 host values: the oracle takes the same values
    want_raw = O.visibility_tri(xp.astype(np.float64), av.faces, fr.astype(np.float64), f32(sc.window_center),
                                float(np.float32(sc.window_half)), sc.depth_res, cull_back=cull_back)
    got_raw = raw.cpu().numpy().view(np.uint32)
    assert np.array_equal(got_raw, want_raw), f"{int((got_raw != want_raw).sum())} words differ"
    want = O.vis_filter(want_raw, knn_v)
    assert np.array_equal(cnt.cpu().numpy(), want)
    assert np.array_equal(cnt_l.cpu().numpy(), want[:, sc.dmap])
    frac = want_raw.size and np.unpackbits(want_raw.view(np.uint8)).mean()
    soft = ((want > 0) & (want < KV)).mean()
    print(f"{name} cull_back={cull_back}: V = 1 for {frac:.3f} of (vertex, direction); "
          f"{soft:.3f} soft (0 < Vbar < 1)")


def test_paper_scale_on_sampled_directions(gpu):
    api = gpu
    sc, xp, knn_v = _inputs("c2_paper")
    av = sc.avatar
    D = sc.frames.shape[0]
    fr = f32(sc.frames.reshape(-1, 9))
    raw = torch.empty(av.Nv, D // 32, dtype=torch.int32, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    cnt = api.avatar_visibility_soft(T(xp.T), T(av.faces, torch.int32), T(fr), sc.window_center, sc.window_half,
                                     sc.depth_res, T(knn_v.T, torch.int32), raw_bits=raw, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    # the oracle on 32 of the 512 directions (each direction is independent)
    sel = np.arange(7, D, D // 32)[:32]
    want_raw = O.visibility_tri(xp.astype(np.float64), av.faces, fr[sel].astype(np.float64),
                                f32(sc.window_center), float(np.float32(sc.window_half)), sc.depth_res)
    got_bits = np.unpackbits(raw.cpu().numpy().view(np.uint8), axis=1, bitorder="little")[:, sel]
    want_bits = np.unpackbits(want_raw.view(np.uint8), axis=1, bitorder="little")[:, :32]
    assert np.array_equal(got_bits, want_bits)
    want = O.vis_filter(want_raw, knn_v)[:, :32]
    assert np.array_equal(cnt.cpu().numpy()[:, sel], want)


def test_soft_shading_matches_oracle(gpu):
    api = gpu
    name = "c1_small"
    sc, xp, knn_v = _inputs(name)
    ref = oracle_frame(name)
    av = sc.avatar
    fr = f32(sc.frames.reshape(-1, 9))
    cnt = O.vis_filter(O.visibility_tri(xp.astype(np.float64), av.faces, fr.astype(np.float64),
                                        f32(sc.window_center), float(np.float32(sc.window_half)), sc.depth_res),
                       knn_v)
    sk = ref["skin"]
    ins = {k: f32(sk[k]) for k in ("xd", "nd", "ag", "rg", "pg", "ubar")}
    skt = {k: T(v.T if v.ndim == 2 else v) for k, v in ins.items()}
    light = dict(L=T(f32(sc.light.L)), A=T(f32(sc.light.A)), w=T(f32(sc.light.w)))
    out = api.avatar_shade(skt, T(av.knn.T, torch.int32), T(cnt[:, sc.dmap], torch.uint8), light,
                           f32(sc.camera.center), vis_den=KV)
    torch.cuda.synchronize()
    col, rad, cull = O.shade_soft(*(ins[k].astype(np.float64) for k in ("xd", "nd", "ag", "rg", "pg", "ubar")),
                                  av.knn, cnt, KV, f32(sc.light.L).astype(np.float64),
                                  f32(sc.light.A).astype(np.float64), f32(sc.light.w).astype(np.float64),
                                  sc.dmap, f32(sc.camera.center).astype(np.float64))
    assert np.array_equal(out["cull"].cpu().numpy(), cull)
    assert rel_err(out["radiance"].cpu().numpy().T, rad) < 5e-5
    assert rel_err(out["color"].cpu().numpy().T, col) < 5e-5


def test_soft_shading_with_saturated_counts_equals_bit_shading(gpu):
    api = gpu
    name = "c3_fd"
    sc = scene(name)
    ref = oracle_frame(name)
    av = sc.avatar
    sk = ref["skin"]
    ins = {k: f32(sk[k]) for k in ("xd", "nd", "ag", "rg", "pg", "ubar")}
    skt = {k: T(v.T if v.ndim == 2 else v) for k, v in ins.items()}
    light = dict(L=T(f32(sc.light.L)), A=T(f32(sc.light.A)), w=T(f32(sc.light.w)))
    bits_l = light_ordered_bits(ref["bits"], sc.dmap)
    V = np.unpackbits(bits_l.view(np.uint8), axis=1, bitorder="little")[:, :len(sc.dmap)]
    knn = T(av.knn.T, torch.int32)
    cam = f32(sc.camera.center)
    a = api.avatar_shade(skt, knn, T(bits_l.view(np.int32), torch.int32), light, cam)
    b = api.avatar_shade(skt, knn, T(V * KV, torch.uint8), light, cam, vis_den=KV)
    gen = torch.Generator(device="cuda").manual_seed(5)
    d_color = torch.rand(a["color"].shape, device="cuda", generator=gen)
    ga = api.avatar_shade_backward(skt, knn, T(bits_l.view(np.int32), torch.int32), light, cam, a, d_color)
    gb = api.avatar_shade_backward(skt, knn, T(V * KV, torch.uint8), light, cam, b, d_color, vis_den=KV)
    torch.cuda.synchronize()
    assert rel_err(b["radiance"].cpu().numpy(), a["radiance"].cpu().numpy()) < 1e-6
    # the two adjoints sum the same per-light terms in different orders (the
    # bit form through its queue of lit lights, the count form lane by lane),
    # each in FP32: about 1e-5 of a gradient's largest element apart
    for k in ("xd", "nd", "ag", "rg", "pg", "ubar", "L"):
        assert rel_err(gb[k].cpu().numpy(), ga[k].cpu().numpy()) < 5e-5, k


def test_unsupported_arguments_are_refused(gpu):
    api = gpu
    from paper_2407_10707_gb300 import _lib as L
    sc, xp, knn_v = _inputs("c3_fd")
    av = sc.avatar
    args = (T(xp.T), T(av.faces, torch.int32), T(f32(sc.frames.reshape(-1, 9))), sc.window_center, sc.window_half)
    with pytest.raises(L.AvatarError):       # beyond the 512^2 depth-map limit
        api.avatar_visibility_soft(*args, 1024, T(knn_v.T, torch.int32))
    with pytest.raises(L.AvatarError):       # an even neighbourhood has no binary median
        api.avatar_visibility_soft(*args, 64, T(knn_v[:, :18].T, torch.int32))


def test_paper_visibility_frame_end_to_end(gpu):
    """The frame with the paper's visibility (Renderer(visibility='paper'))
    against the oracle chain skin -> triangle-ID visibility -> filters -> soft
    shading -> projection -> brute-force compositing."""
    api = gpu
    from paper_2407_10707_gb300 import render
    from oracle import pipeline as OP
    name = "c1_small"
    sc = scene(name)
    av = sc.avatar
    knn_v = synth.vertex_knn(av.xv, KV)
    bone = O.fk(av.parents, av.joints, av.pose)
    sk = O.skin(av, bone)
    fr = f32(sc.frames.reshape(-1, 9))
    cnt = O.vis_filter(O.visibility_tri(f32(sk["xp"]).astype(np.float64), av.faces, fr.astype(np.float64),
                                        f32(sc.window_center), float(np.float32(sc.window_half)), sc.depth_res,
                                        cull_back=True), knn_v)
    col, _, cull = O.shade_soft(sk["xd"], sk["nd"], sk["ag"], sk["rg"], sk["pg"], sk["ubar"], av.knn, cnt, KV,
                                sc.light.L, sc.light.A, sc.light.w, sc.dmap, sc.camera.center)
    pr = O.project(sk["xd"], sk["cov"], av.opacity, cull, sc.camera)
    cam = sc.camera
    rgb, _, _, amb = O.composite(pr["mean2d"], pr["conic"], av.opacity, col, pr["depth"], pr["valid"], cam.width,
                                 cam.height)
    st = render.scene_tensors(sc)
    r = render.Renderer(st, visibility="paper", knn_v=T(knn_v.T, torch.int32))
    img = r.forward().cpu().numpy().reshape(3, -1).T
    r.check()
    ok = amb == 0
    bad = np.abs(img - rgb).max(axis=1) > 2e-4
    print(f"paper visibility frame: {int((bad & ok).sum())} pixels > 2e-4 of {len(bad)}")
    assert (bad & ok).mean() < 0.01
    assert np.abs(img - rgb).max() < 0.05
    # and the training step runs through the soft visibility
    ts = render.TrainStep(st, r.sb.image.clone() * 0.9, visibility="paper", knn_v=T(knn_v.T, torch.int32))
    torch.cuda.synchronize()
    ts.check()
    g = ts.grads()
    assert all(bool(torch.isfinite(v).all()) for v in g.values())
    assert float(g["L"].abs().sum()) > 0
