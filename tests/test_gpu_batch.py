"""The batched render (avatar_render_batch): poses x cameras of mixed
resolution, each pose with its own light, one launch per stage.

Every stage of the batch runs the same per-element arithmetic as the
per-frame calls, and the one depth sort over all views keeps each view's
(depth, index) order, so each view's image must equal the per-frame render of
that view bit for bit.  Gradients are sums over views of the per-frame
gradients (the batch loss is the mean over all views' pixels), equal up to the
order of floating-point accumulation: 2e-4 relative.  Against the FP64
oracle, views are checked stage by stage through their per-frame renders
(tests/_chain.py), at test size and at the full C4 configuration.
"""
import dataclasses

import numpy as np
import pytest

from _common import rel_err, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PIX_TOL = 2e-4
GRAD_TOL = 2e-4


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    from paper_2407_10707_gb300 import api, render
    return api, render


@pytest.fixture(scope="module")
def batch():
    return synth.config_batch("c4_small")


def view_scene(b, v):
    """The single-frame scene of view v: its pose, its pose's light, its camera."""
    p = int(b.view_pose[v])
    sc = b.scene
    av = dataclasses.replace(sc.avatar, pose=b.poses[p])
    light = dataclasses.replace(sc.light, L=b.lights[p])
    return dataclasses.replace(sc, avatar=av, light=light, camera=b.cameras[v])


def N(t):
    return t.detach().float().cpu().numpy()


@pytest.mark.parametrize("attr_dtype", ["f32", "bf16"])
def test_batch_images_equal_per_frame_renders(gpu, batch, attr_dtype):
    api, render = gpu
    br = render.BatchRenderer(batch, tile=16, attr_dtype=attr_dtype)
    for v in range(batch.V):
        r = render.Renderer(render.scene_tensors(view_scene(batch, v), attr_dtype=attr_dtype))
        r.check()
        diff = (br.image(v) - r.sb.image).abs()
        assert torch.equal(br.image(v), r.sb.image), \
            f"view {v}: {int((diff > 0).sum())} of {diff.numel()} values differ, max {float(diff.max()):.3e}"


def test_batch_views_meet_the_oracle_stage_by_stage(gpu, batch):
    """Views 0 (64 x 64) and 3 (100 x 72) equal their per-frame renders bit
    for bit, and those meet the FP64 oracle stage by stage on every pixel
    (tests/_chain.py): no exemption beyond the pixels the oracle flags."""
    from _chain import chain_check
    api, render = gpu
    br = render.BatchRenderer(batch, tile=16)
    for v in (0, 3):
        sc = view_scene(batch, v)
        r = render.Renderer(render.scene_tensors(sc), tile=16)
        torch.cuda.synchronize()
        r.check()
        assert torch.equal(r.sb.image, br.image(v))
        rep = chain_check(r, sc)
        rep.pop("gpu")
        print(f"view {v}:", rep)


def _targets(br, seed=3):
    rng = np.random.default_rng(seed)
    img = N(br.images)
    return torch.as_tensor(np.clip(img * rng.uniform(0.8, 1.2, img.shape), 0, None).astype(np.float32),
                           device="cuda")


def test_batch_gradients_are_the_sum_of_per_frame_gradients(gpu, batch):
    api, render = gpu
    probe = render.BatchRenderer(batch, tile=16)
    targets = _targets(probe)
    br = render.BatchRenderer(batch, targets=targets, tile=16)
    loss_b = float(br.loss.item())
    gb = {k: N(v) for k, v in br.grads.items()}
    total = float(br.offsets[-1])
    want = {k: np.zeros_like(v) for k, v in gb.items()}
    loss_sum = 0.0
    for v in range(batch.V):
        h, w = br.sizes[v]
        tgt = targets[br.offsets[v]:br.offsets[v + 1]].view(3, h, w)
        ts = render.TrainStep(render.scene_tensors(view_scene(batch, v)), tgt)
        torch.cuda.synchronize()
        ts.check()
        wgt = 3 * h * w / total
        loss_sum += wgt * float(ts.loss.item())
        g = {k: N(x) for k, x in ts.grads().items()}
        for k in ("xg", "logscale", "quat", "opacity", "wv", "av", "rv", "pv"):
            want[k] += wgt * g[k]
        want["L"][int(batch.view_pose[v])] += wgt * g["L"]
    assert abs(loss_b - loss_sum) < 1e-5 * abs(loss_sum)
    for k in want:
        e = rel_err(gb[k], want[k])
        assert e < GRAD_TOL, f"{k}: relative error {e}"


def test_batch_graph_replay_is_identical(gpu, batch):
    api, render = gpu
    probe = render.BatchRenderer(batch, tile=16)
    br = render.BatchRenderer(batch, targets=_targets(probe), tile=16)
    img0 = br.images.clone()
    g0 = {k: v.clone() for k, v in br.grads.items()}
    br.capture()
    br.images.zero_()
    br.replay()
    br.replay()
    torch.cuda.synchronize()
    br.check()
    assert torch.equal(br.images, img0)
    for k, v in g0.items():
        assert rel_err(N(br.grads[k]), N(v)) < 1e-5, k   # atomics may add in another order


def test_batch_images_do_not_depend_on_region_masks(gpu, batch):
    """The batch's pair keys with and without region masks give the same
    images bit for bit (AVATAR_TUNE_REGION_MASKS, the form past 2^24 tiles)."""
    api, render = gpu
    from paper_2407_10707_gb300 import _lib as L
    lib, ctx = L.load(), api.context()
    imgs = []
    try:
        for masks in (1, 0):
            assert lib.avatar_ctx_set_tuning(ctx, L.TUNE_REGION_MASKS, masks) == 0
            br = render.BatchRenderer(batch, tile=32)
            torch.cuda.synchronize()
            br.check()
            imgs.append(br.images.clone())
    finally:
        lib.avatar_ctx_set_tuning(ctx, L.TUNE_REGION_MASKS, 1)
    assert torch.equal(imgs[0], imgs[1])


def test_pair_overflow_is_reported(gpu, batch):
    api, render = gpu
    from paper_2407_10707_gb300 import _lib as L
    with pytest.raises(L.AvatarError) as e:
        render.BatchRenderer(batch, tile=16, pair_capacity=1000)
    assert e.value.code == 3


def test_autotune_keeps_the_images(gpu, batch):
    api, render = gpu
    probe = render.BatchRenderer(batch, tile=16)
    br = render.BatchRenderer(batch, targets=_targets(probe), tile=0)
    img0 = br.images.clone()
    tile, ppt, bppt = br.autotune()
    assert tile in (8, 16, 32) and ppt in (1, 2, 4) and bppt in (1, 2, 4)
    br.status.zero_()
    br.step()
    torch.cuda.synchronize()
    br.check()
    print(f"autotuned: tile {tile}, blend pixels/thread {ppt}, backward pixels/thread {bppt}")
    assert torch.equal(br.images, img0)   # the image does not depend on the tile edge or the split
    lib = L_lib()
    for key, want in ((2, 16), (0, 1), (1, 1)):   # restore the defaults for later tests
        lib.avatar_ctx_set_tuning(api.context(), key, want)


def L_lib():
    from paper_2407_10707_gb300 import _lib as L
    return L.load()


def test_full_c4_batch_bf16_matches_oracle_stage_by_stage(gpu):
    """The C4 batch as the benchmark runs it - 32 poses x 4 cameras at 512^2,
    1080^2 and 1920 x 1080, the 200k-Gaussian avatar with a light per pose,
    BF16 attribute storage, Gaussians in nearest-vertex order, faces by
    normal within raster chunks, autotuned tile
    edge and pixel splits.  A 1080^2 and a 1920 x 1080 view equal, bit for
    bit, the per-frame renders of those views with the same choices, and each
    per-frame render meets the FP64 oracle stage by stage (tests/_chain.py)
    on 4,096 sampled pixels, the oracle run on the BF16-rounded avatar in the
    same order: only the pixels the oracle flags ambiguous are excluded."""
    from _chain import chain_check
    from _common import bf16_scene
    api, render = gpu
    b = synth.config_batch("c4_batch")
    forder = synth.face_normal_order(b.scene.avatar.xv, b.scene.avatar.faces)
    br = render.BatchRenderer(b, tile=0, attr_dtype="bf16", spatial_order=True, face_order=forder)
    lib = L_lib()
    try:
        tile, ppt, bppt = br.autotune()
        br.status.zero_()
        br.forward()
        torch.cuda.synchronize()
        br.check()
        np_order = synth.nearest_vertex_order(b.scene)
        assert np.array_equal(br.order.cpu().numpy(), np_order)
        rng = np.random.default_rng(11)
        for v in (1, 2):
            scv = view_scene(b, v)
            stv, _ = render.spatially_ordered(render.scene_tensors(scv, attr_dtype="bf16"))
            stv, _ = render.faces_ordered(stv, forder)
            rv = render.Renderer(stv, tile=tile)
            torch.cuda.synchronize()
            rv.check()
            assert torch.equal(rv.sb.image, br.image(v)), f"view {v} differs from its per-frame render"
            n = scv.camera.width * scv.camera.height
            pix = np.sort(rng.choice(n, size=4096, replace=False)).astype(np.int32)
            rep = chain_check(rv, bf16_scene(synth.permute_faces(synth.permute_gaussians(scv, np_order), forder)),
                              pixels=pix)
            rep.pop("gpu")
            print(f"view {v} ({scv.camera.width}x{scv.camera.height}), tile {tile}, blend split {ppt}:", rep)
            del rv
    finally:
        for key, want in ((2, 16), (0, 1), (1, 1)):   # restore the defaults for later tests
            lib.avatar_ctx_set_tuning(api.context(), key, want)
