"""The image loss of Eq. 5 on the GPU (avatar_image_loss) against the FP64
oracle: (1 - lambda) L1 + lambda D-SSIM, 11 x 11 Gaussian window.

FP32 windowed sums of 121 terms: the loss within 1e-5 relative; the gradient
within 1e-4 of its largest magnitude (per-element FP32 chains of ~250 terms).
"""
import numpy as np
import pytest

from _common import rel_err

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


@pytest.mark.parametrize("shape,lam", [((3, 64, 80), 0.2), ((3, 130, 97), 0.2), ((1, 33, 40), 1.0),
                                       ((3, 40, 33), 0.0)])
def test_image_loss_matches_oracle(gpu, shape, lam):
    api = gpu
    from oracle import ssim as S
    rng = np.random.default_rng(sum(shape))
    x = rng.uniform(0, 1, size=shape).astype(np.float32)
    y = np.clip(x + rng.normal(0, 0.15, shape), 0, 1).astype(np.float32)
    loss, d = api.avatar_image_loss(torch.as_tensor(x, device="cuda"), torch.as_tensor(y, device="cuda"), lam)
    torch.cuda.synchronize()
    want, g = S.image_loss_grad(x.astype(np.float64), y.astype(np.float64), lam)
    got = float(loss.item())
    print(f"{shape} lambda={lam}: loss {got:.7f} vs {want:.7f}, grad rel err {rel_err(d.cpu().numpy(), g):.2e}")
    assert abs(got - want) < 1e-5 * abs(want)
    assert rel_err(d.cpu().numpy(), g) < 1e-4


def test_l1_part_equals_the_l1_loss_and_batches_accumulate(gpu):
    api = gpu
    rng = np.random.default_rng(5)
    x = torch.as_tensor(rng.uniform(0, 1, (3, 50, 70)).astype(np.float32), device="cuda")
    y = torch.as_tensor(rng.uniform(0, 1, (3, 50, 70)).astype(np.float32), device="cuda")
    l_img, d_img = api.avatar_image_loss(x, y, 0.0)
    l_l1, d_l1 = api.avatar_l1_loss(x, y)
    torch.cuda.synchronize()
    assert abs(float(l_img.item()) - float(l_l1.item())) < 1e-6
    assert torch.allclose(d_img, d_l1.view_as(d_img), atol=1e-12)
    # two weighted, accumulated calls give the weighted sum of the losses
    acc = torch.zeros(1, device="cuda")
    api.avatar_image_loss(x, y, 0.2, loss=acc, weight=0.25, accumulate=True, want_grad=False)
    api.avatar_image_loss(y, x, 0.2, loss=acc, weight=0.75, accumulate=True, want_grad=False)
    a, _ = api.avatar_image_loss(x, y, 0.2, want_grad=False)
    b, _ = api.avatar_image_loss(y, x, 0.2, want_grad=False)
    torch.cuda.synchronize()
    assert abs(float(acc.item()) - (0.25 * float(a.item()) + 0.75 * float(b.item()))) < 1e-6


def test_train_step_with_the_paper_image_loss_matches_fp64_adjoint(gpu):
    """TrainStep's default loss is Eq. 5's (lambda 0.2): its gradients against
    the FP64 adjoint of the frame with the FP64 image loss, 1e-3 relative."""
    api = gpu
    from oracle import adjoint as AJ
    from oracle import ssim as S
    from paper_2407_10707_gb300 import render
    from _common import oracle_frame, scene
    sc = scene("c3_fd")
    ref = oracle_frame("c3_fd")
    av = sc.avatar
    rng = np.random.default_rng(6)
    target = np.clip(ref["rgb"] * rng.uniform(0.8, 1.2, ref["rgb"].shape), 0, None)
    fixed = dict(knn=av.knn, xv=AJ.t64(av.xv), dxv=AJ.t64(av.dxv), nv=AJ.t64(av.nv), bone=AJ.t64(ref["bone"]),
                 bits=ref["bits"], dmap=sc.dmap, A=AJ.t64(sc.light.A), w=AJ.t64(sc.light.w),
                 cam_center=AJ.t64(sc.camera.center), culled=ref["cull"], valid=ref["proj"]["valid"], cam=sc.camera)
    params = dict(xg=av.xg, logscale=av.logscale, quat=av.quat, opacity=av.opacity, av=av.av, rv=av.rv, pv=av.pv,
                  L=sc.light.L, wv=av.wv)
    tp = {k: AJ.t64(v).requires_grad_(True) for k, v in params.items()}
    img = AJ.render(tp, fixed)                                          # [H, W, 3]
    tgt64 = AJ.t64(target).reshape(img.shape)
    loss_ref = S.image_loss_torch(img.permute(2, 0, 1), tgt64.permute(2, 0, 1), 0.2)
    loss_ref.backward()
    st = render.scene_tensors(sc)
    W, H = sc.camera.width, sc.camera.height
    tgt = torch.as_tensor(np.asarray(target, np.float32).T.reshape(3, H, W).copy(), device="cuda")
    ts = render.TrainStep(st, tgt)
    torch.cuda.synchronize()
    ts.check()
    assert abs(float(ts.loss.item()) - float(loss_ref)) < 1e-3 * float(loss_ref)
    g = {k: v.detach().cpu().numpy() for k, v in ts.grads().items()}
    for k in ("xg", "logscale", "quat", "opacity", "av", "rv", "pv", "L", "wv"):
        got = g[k].T if g[k].ndim == 2 and k not in ("L", "wv") else g[k]
        e = rel_err(got, tp[k].grad.numpy())
        assert e < 1e-3, f"{k}: relative error {e}"
