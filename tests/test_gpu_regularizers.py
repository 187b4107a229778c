"""The regularisers of Sec. 3.3 on the GPU (avatar_regularizers) against the
FP64 oracle: the four sums within 1e-5 relative (FP32 terms, FP64 sums) and
every gradient within 1e-5 of its largest magnitude."""
import numpy as np
import pytest

from _common import rel_err, scene, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    from paper_2407_10707_gb300 import api
    return api


@pytest.mark.parametrize("name,dx", [("c1_small", 0.0), ("c3_fd", 0.01)])
def test_regularizers_match_oracle(gpu, name, dx):
    api = gpu
    from oracle import regularizers as RG
    sc = scene(name)
    av = sc.avatar
    rng = np.random.default_rng(3)
    dxv = (dx * rng.normal(size=av.xv.shape)).astype(np.float32)
    logscale = (av.logscale + rng.normal(0, 0.6, av.logscale.shape)).astype(np.float32)  # some above s0
    knn_v = synth.vertex_knn(av.xv, 19)
    t = api.avatar_tensors(av)
    t["dxv"] = torch.as_tensor(dxv.T.copy(), device="cuda")
    t["logscale"] = torch.as_tensor(logscale.T.copy(), device="cuda")
    grads = {k: torch.zeros_like(t[k]) for k in ("xg", "logscale", "av", "rv", "pv", "dxv")}
    loss, terms = api.avatar_regularizers(t, torch.as_tensor(knn_v.T.copy(), dtype=torch.int32, device="cuda"),
                                          grads=grads)
    torch.cuda.synchronize()
    f = lambda a: np.asarray(a, np.float32).astype(np.float64)
    total, want, g = RG.regularizers(f(av.xg), f(logscale), av.knn, f(av.xv), f(av.av), f(av.rv), f(av.pv), knn_v,
                                     f(dxv))
    got = terms.cpu().numpy()
    for i, k in enumerate(("smooth", "mdist", "disp", "scale")):
        assert abs(got[i] - want[k]) <= 1e-5 * max(abs(want[k]), 1e-12), k
    assert abs(float(loss.item()) - total) < 1e-5 * total
    for k in grads:
        gg = grads[k].cpu().numpy()
        gg = gg.T if gg.ndim == 2 else gg
        assert rel_err(gg, g[k]) < 1e-5, k


def test_gradients_accumulate_into_the_buffers(gpu):
    api = gpu
    av = scene("c3_fd").avatar
    knn_v = torch.as_tensor(synth.vertex_knn(av.xv, 19).T.copy(), dtype=torch.int32, device="cuda")
    t = api.avatar_tensors(av)
    g1 = {"av": torch.zeros_like(t["av"])}
    api.avatar_regularizers(t, knn_v, grads=g1)
    g2 = {"av": torch.full_like(t["av"], 0.5)}
    api.avatar_regularizers(t, knn_v, grads=g2)
    torch.cuda.synchronize()
    assert torch.allclose(g2["av"], g1["av"] + 0.5, atol=1e-6)


def test_train_step_with_regularizers_matches_fp64_adjoint(gpu):
    """TrainStep(regularize=True): the L1 image loss plus the regularisers,
    against one FP64 autograd graph of both, 1e-3 relative."""
    api = gpu
    from oracle import adjoint as AJ
    from oracle import regularizers as RG
    from paper_2407_10707_gb300 import render
    from _common import oracle_frame
    sc = scene("c3_fd")
    ref = oracle_frame("c3_fd")
    av = sc.avatar
    knn_v = synth.vertex_knn(av.xv, 19)
    rng = np.random.default_rng(8)
    target = np.clip(ref["rgb"] * rng.uniform(0.8, 1.2, ref["rgb"].shape), 0, None)
    fixed = dict(knn=av.knn, xv=AJ.t64(av.xv), dxv=AJ.t64(av.dxv), nv=AJ.t64(av.nv), bone=AJ.t64(ref["bone"]),
                 bits=ref["bits"], dmap=sc.dmap, A=AJ.t64(sc.light.A), w=AJ.t64(sc.light.w),
                 cam_center=AJ.t64(sc.camera.center), culled=ref["cull"], valid=ref["proj"]["valid"], cam=sc.camera)
    params = dict(xg=av.xg, logscale=av.logscale, quat=av.quat, opacity=av.opacity, av=av.av, rv=av.rv, pv=av.pv,
                  L=sc.light.L, wv=av.wv)
    tp = {k: AJ.t64(v).requires_grad_(True) for k, v in params.items()}
    img = AJ.render(tp, fixed)
    terms = RG.terms_torch(tp["xg"], tp["logscale"], av.knn, fixed["xv"], tp["av"], tp["rv"], tp["pv"], knn_v,
                           fixed["dxv"])
    loss = AJ.l1_loss(img, AJ.t64(target).reshape(img.shape)) + sum(RG.WEIGHTS[k] * terms[k] for k in terms)
    loss.backward()
    st = render.scene_tensors(sc)
    W, H = sc.camera.width, sc.camera.height
    tgt = torch.as_tensor(np.asarray(target, np.float32).T.reshape(3, H, W).copy(), device="cuda")
    ts = render.TrainStep(st, tgt, ssim_weight=0.0, regularize=True,
                          knn_v=torch.as_tensor(knn_v.T.copy(), dtype=torch.int32, device="cuda"))
    torch.cuda.synchronize()
    ts.check()
    assert abs(float(ts.loss.item()) - float(loss)) < 1e-4 * float(loss)
    g = {k: v.detach().cpu().numpy() for k, v in ts.grads().items()}
    for k in ("xg", "logscale", "quat", "opacity", "av", "rv", "pv", "L", "wv"):
        got = g[k].T if g[k].ndim == 2 and k not in ("L", "wv") else g[k]
        e = rel_err(got, tp[k].grad.numpy())
        assert e < 1e-3, f"{k}: relative error {e}"
