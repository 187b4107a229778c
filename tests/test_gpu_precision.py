"""The precision form: BF16 attribute storage and tensor-core shading.

* BF16 storage (albedo, roughness, tint, opacity, log-scale, rotation): the
  arithmetic stays FP32, so the frame must match the FP64 oracle run on the
  BF16-rounded attribute values at the FP32 tolerances; the error that the
  rounding itself causes (against the oracle on the FP32 values) is reported.
* Tensor-core shading (BF16 weights D, S; FP32 accumulation): colours within
  1e-3 max-abs of the oracle, and images within 1e-3 max-abs of the plain
  FP32 CUDA-core frame on the same GPU (pixels are convex combinations of
  colours, so the colour bound carries over).
"""
import numpy as np
import pytest

from _common import BF16_ATTRS, OP, bf16_scene, f32, light_ordered_bits, oracle_frame, rel_err, scene

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PIX_TOL = 2e-4
TC_TOL = 1e-3


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    from paper_2407_10707_gb300 import api, render
    return api, render


def N(t):
    return t.detach().float().cpu().numpy()


@pytest.mark.parametrize("name", ["c1_small", "c3_fd"])
def test_bf16_storage_frame_matches_oracle_on_rounded_attributes(gpu, name):
    api, render = gpu
    sc = scene(name)
    scb = bf16_scene(sc)
    ref = OP.frame(scb)
    st = render.scene_tensors(sc, attr_dtype="bf16")
    t = st["avatar"]
    for k in BF16_ATTRS:   # the device conversion rounds exactly as the oracle's inputs were rounded
        assert t[k].dtype == torch.bfloat16
        want = getattr(scb.avatar, k)
        assert np.array_equal(N(t[k]).T if want.ndim == 2 else N(t[k]), want.astype(np.float32)), k
    r = render.Renderer(st)
    img = N(r.forward()).reshape(3, -1).T
    r.check()
    sk = ref["skin"]
    assert rel_err(N(r.sk["xd"]).T, sk["xd"]) < 1e-5
    assert rel_err(N(r.sk["cov"]).T, sk["cov"]) < 5e-5
    assert rel_err(N(r.sk["ag"]).T, sk["ag"]) < 1e-5
    assert rel_err(N(r.sk["rg"]), sk["rg"]) < 1e-5
    ok = ref["amb"] == 0
    bad = np.abs(img - ref["rgb"]).max(axis=1) > PIX_TOL
    assert (bad & ok).mean() < 0.01
    quant = np.abs(img - oracle_frame(name)["rgb"])
    print(f"{name}: BF16 storage vs oracle on rounded inputs: {int((bad & ok).sum())} pixels > {PIX_TOL}; "
          f"rounding effect vs FP32-stored oracle: max {quant.max():.2e}, mean {quant.mean():.2e}")


@pytest.mark.parametrize("name", ["c1_small", "c3_fd"])
def test_tensor_core_shading_frame(gpu, name):
    api, render = gpu
    sc = scene(name)
    ref = oracle_frame(name)
    st = render.scene_tensors(sc)
    r32 = render.Renderer(st)
    img32 = N(r32.forward()).reshape(3, -1).T
    rtc = render.Renderer(st, shade_tc=True)
    imgtc = N(rtc.forward()).reshape(3, -1).T
    r32.check()
    rtc.check()
    assert np.array_equal(N(rtc.sh["cull"]), N(r32.sh["cull"]))
    col_err = np.abs(N(rtc.sh["color"]) - N(r32.sh["color"])).max()
    rad_err = rel_err(N(rtc.sh["radiance"]), N(r32.sh["radiance"]))
    img_err = np.abs(imgtc - img32).max()
    ok = ref["amb"] == 0
    bad = np.abs(imgtc - ref["rgb"]).max(axis=1) > TC_TOL
    print(f"{name}: tensor-core vs FP32 shading: colour {col_err:.2e}, radiance rel {rad_err:.2e}, "
          f"image {img_err:.2e}; {int((bad & ok).sum())} pixels > {TC_TOL} vs oracle")
    assert col_err < TC_TOL
    assert img_err < TC_TOL
    assert (bad & ok).mean() < 0.01


def test_bf16_tensor_core_train_step_gradients(gpu):
    """BF16 storage + tensor-core forward shading + FP32 backward: gradients
    against the FP64 adjoint of the BF16-rounded problem."""
    api, render = gpu
    from oracle import adjoint as AJ
    sc = scene("c3_fd")
    scb = bf16_scene(sc)
    ref = OP.frame(scb)
    av = scb.avatar
    rng = np.random.default_rng(5)
    target = np.clip(ref["rgb"] * rng.uniform(0.8, 1.2, ref["rgb"].shape), 0, None)
    fixed = dict(knn=av.knn, xv=AJ.t64(av.xv), dxv=AJ.t64(av.dxv), nv=AJ.t64(av.nv), bone=AJ.t64(ref["bone"]),
                 bits=ref["bits"], dmap=scb.dmap, A=AJ.t64(scb.light.A), w=AJ.t64(scb.light.w),
                 cam_center=AJ.t64(scb.camera.center), culled=ref["cull"], valid=ref["proj"]["valid"],
                 cam=scb.camera)
    params = dict(xg=av.xg, logscale=av.logscale, quat=av.quat, opacity=av.opacity, av=av.av, rv=av.rv, pv=av.pv,
                  L=scb.light.L, wv=av.wv)
    tp = {k: AJ.t64(v).requires_grad_(True) for k, v in params.items()}
    img = AJ.render(tp, fixed)
    loss_ref = AJ.l1_loss(img, AJ.t64(target).reshape(img.shape))
    loss_ref.backward()
    st = render.scene_tensors(sc, attr_dtype="bf16")
    W, H = sc.camera.width, sc.camera.height
    tgt = torch.as_tensor(f32(target).T.reshape(3, H, W).copy(), device="cuda")
    ts = render.TrainStep(st, tgt, shade_tc=True, ssim_weight=0.0)
    loss = float(ts.step().item())
    torch.cuda.synchronize()
    ts.check()
    g = {k: N(v) for k, v in ts.grads().items()}
    worst = {}
    for k in ("xg", "logscale", "quat", "opacity", "av", "rv", "pv", "L", "wv"):
        got = g[k].T if g[k].ndim == 2 and k not in ("L", "wv") else g[k]
        worst[k] = rel_err(got, tp[k].grad.numpy())
    print("BF16 + tensor-core train step: loss rel err %.2e; grad rel err %s" % (
        abs(loss - float(loss_ref)) / float(loss_ref), {k: f"{v:.1e}" for k, v in worst.items()}))
    assert abs(loss - float(loss_ref)) < 2e-3 * float(loss_ref)
    for k, e in worst.items():
        assert e < 1e-2, f"{k}: relative error {e}"
