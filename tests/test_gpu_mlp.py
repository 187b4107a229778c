"""The displacement MLP of Sec. 3.1 on the tensor cores (avatar_mlp) against
the oracle.

Tolerances.  The kernel rounds the same values to bfloat16 as the oracle's
bf16 mode, but it forms the Fourier phases and every layer's sums in FP32
where the oracle uses FP64 (and takes the hardware sine and cosine after an
exact range reduction, absolute error about 4e-7, below the FP32 error of
the phase); a value lying within that error of a bfloat16 rounding boundary
rounds the other way, one bfloat16 step (2^-8 relative) in one feature or
activation.  An FP32 emulation of the kernel's
arithmetic on 4000 points of these weights puts the effect at 0.55 % of the
output's RMS at worst and 3e-5 of it on average; the bounds below are about
four times those (2 % worst, 2e-4 mean).  Against the plain FP64 network the
bfloat16 operands themselves dominate (1.3 % worst, 0.26 % mean on the same
points): bounded at 5 % and 1 %."""
import numpy as np
import pytest

from _common import scene, synth

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


def _oracle(x, theta, w, bf):
    from oracle import mlp as M
    f = lambda a: np.asarray(a, np.float32).astype(np.float64)  # the kernel's FP32 inputs
    return M.forward(f(x), f(theta), f(w["Bf"]), f(w["W1"]), f(w["b1"]), f(w["W2"]), f(w["b2"]), f(w["W3"]),
                     f(w["b3"]), f(w["W4"]), f(w["b4"]), bf=bf)


def _run(api, x, theta, w, status=None):
    wt = api.mlp_tensors(w, "cuda")
    xt = torch.as_tensor(np.asarray(x, np.float32).T.copy(), device="cuda")
    th = np.asarray(theta, np.float32)
    tt = torch.as_tensor(th.reshape(th.shape[0], -1) if th.ndim == 2 else th.ravel(), device="cuda")
    dx = api.avatar_mlp(xt, tt, wt, status=status)
    torch.cuda.synchronize()
    return dx.cpu().numpy().T.astype(np.float64)


def _check(got, x, theta, w):
    want = _oracle(x, theta, w, bf=True)
    full = _oracle(x, theta, w, bf=False)
    rms = np.sqrt((want ** 2).mean())
    d = np.abs(got - want)
    assert d.max() <= 2e-2 * rms and d.mean() <= 2e-4 * rms, (d.max() / rms, d.mean() / rms)
    e = np.abs(got - full)
    assert e.max() <= 5e-2 * rms and e.mean() <= 1e-2 * rms, (e.max() / rms, e.mean() / rms)


@pytest.mark.parametrize("n,p", [(1000, 72), (128, 72), (127, 72), (1, 72), (300, 0), (513, 128)])
def test_mlp_matches_oracle(gpu, n, p):
    api = gpu
    rng = np.random.default_rng(n + p)
    w = synth.mlp_weights(p, pose_dims=p)
    x = rng.uniform(-1.0, 1.0, size=(n, 3))
    theta = rng.normal(0.0, 0.3, size=p)
    st = api.status_word("cuda")
    got = _run(api, x, theta, w, status=st)
    assert int(st.item()) == 0
    _check(got, x, theta, w)


def test_mlp_on_avatar_vertices_full_size(gpu):
    """The 50k-vertex avatar at its own pose, 2000 sampled rows checked."""
    api = gpu
    sc = scene("c2_paper")
    av = sc.avatar
    w = synth.mlp_weights(1)
    theta = av.pose.ravel()
    got = _run(api, av.xv, theta, w)
    rows = np.random.default_rng(5).choice(av.xv.shape[0], 2000, replace=False)
    _check(got[rows], av.xv[rows], theta, w)


def test_rows_do_not_depend_on_the_batch(gpu):
    """Each row's result is the same bits whatever the number of points and
    wherever the row falls in the persistent schedule."""
    api = gpu
    rng = np.random.default_rng(9)
    w = synth.mlp_weights(2)
    x = rng.uniform(-1.0, 1.0, size=(40_000, 3))
    theta = rng.normal(0.0, 0.3, size=72)
    a = _run(api, x, theta, w)
    b = _run(api, x[:1000], theta, w)
    c = _run(api, x[39_000:], theta, w)
    assert np.array_equal(a[:1000], b) and np.array_equal(a[39_000:], c)


def test_empty_and_invalid(gpu):
    api = gpu
    from paper_2407_10707_gb300 import _lib as L
    w = api.mlp_tensors(synth.mlp_weights(0), "cuda")
    x = torch.empty(3, 0, device="cuda")
    dx = api.avatar_mlp(x, torch.zeros(72, device="cuda"), w)
    assert dx.shape == (3, 0)
    with pytest.raises(L.AvatarError):
        api.avatar_mlp(torch.zeros(3, 4, device="cuda"), torch.zeros(129, device="cuda"),
                       api.mlp_tensors(synth.mlp_weights(0, pose_dims=129), "cuda"))


def test_renderer_evaluates_the_mlp_before_skinning(gpu):
    """A frame rendered with the MLP is bit-identical to the frame rendered
    with the MLP's output supplied as the avatar's fixed displacement, and it
    differs from the frame without displacement."""
    api = gpu
    from paper_2407_10707_gb300 import render
    sc = scene("c1_small")
    w = api.mlp_tensors(synth.mlp_weights(4), "cuda")
    st = render.scene_tensors(sc, "cuda")
    r_mlp = render.Renderer(st, mlp=w)
    img_mlp = r_mlp.forward().clone()
    r_mlp.check()
    dx = api.avatar_mlp(st["avatar"]["xv"], st["avatar"]["pose"].reshape(-1), w)
    st2 = render.scene_tensors(sc, "cuda")
    st2["avatar"]["dxv"].copy_(dx)
    img_fixed = render.Renderer(st2).forward().clone()
    st3 = render.scene_tensors(sc, "cuda")
    st3["avatar"]["dxv"].zero_()
    img_zero = render.Renderer(st3).forward().clone()
    torch.cuda.synchronize()
    assert torch.equal(img_mlp, img_fixed)
    assert float(dx.abs().max()) > 1e-4 and not torch.equal(img_mlp, img_zero)


@pytest.mark.parametrize("n,T", [(1000, 5), (300, 4), (513, 7), (128, 2)])
def test_mlp_mean_over_poses_matches_oracle(gpu, n, T):
    """The mean displacement over T poses (Sec. 4's average over the training
    poses): the oracle's mean of the per-pose networks, with the per-pose
    bounds scaled by the per-pose RMS."""
    api = gpu
    rng = np.random.default_rng(n * 7 + T)
    w = synth.mlp_weights(3)
    x = rng.uniform(-1.0, 1.0, size=(n, 3))
    poses = rng.normal(0.0, 0.3, size=(T, 72))
    st = api.status_word("cuda")
    got = _run(api, x, poses, w, status=st)
    assert int(st.item()) == 0
    per = [_oracle(x, th, w, bf=True) for th in poses]
    want = np.mean(per, axis=0)
    rms = np.sqrt(np.mean([np.mean(p ** 2) for p in per]))
    d = np.abs(got - want)
    assert d.max() <= 2e-2 * rms and d.mean() <= 2e-4 * rms, (d.max() / rms, d.mean() / rms)


def test_average_displacement_sets_the_avatar_displacement(gpu):
    api = gpu
    from paper_2407_10707_gb300 import render
    sc = scene("c1_small")
    st = render.scene_tensors(sc, "cuda")
    w = api.mlp_tensors(synth.mlp_weights(5), "cuda")
    poses = torch.as_tensor(np.random.default_rng(2).normal(0, 0.3, size=(6, 24, 3)), dtype=torch.float32,
                            device="cuda")
    dx = render.average_displacement(st, w, poses)
    want = api.avatar_mlp(st["avatar"]["xv"], poses.reshape(6, 72), w)
    torch.cuda.synchronize()
    assert dx.data_ptr() == st["avatar"]["dxv"].data_ptr() and torch.equal(dx, want)
    r = render.Renderer(st)
    r.forward()
    r.check()


def test_mlp_many_poses_on_one_tile(gpu):
    """100 points (one tile, one CTA) averaged over 300 poses: one CTA walks
    a long list of (tile, pose) items through both slots."""
    api = gpu
    rng = np.random.default_rng(17)
    w = synth.mlp_weights(6)
    x = rng.uniform(-1.0, 1.0, size=(100, 3))
    poses = rng.normal(0.0, 0.3, size=(300, 72))
    got = _run(api, x, poses, w)
    per = [_oracle(x, th, w, bf=True) for th in poses]
    want = np.mean(per, axis=0)
    rms = np.sqrt(np.mean([np.mean(p ** 2) for p in per]))
    d = np.abs(got - want)
    assert d.max() <= 2e-2 * rms and d.mean() <= 2e-4 * rms, (d.max() / rms, d.mean() / rms)
