"""The Gaussians' storage order (avatar_gaussian_order, avatar_gather_columns)
through the C ABI: the order is the stable sort by nearest vertex, bit for
bit; the gather is numpy's fancy indexing; a frame of the reordered avatar
meets the oracle run on the same reordered avatar, stage by stage."""
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
    from paper_2407_10707_gb300 import api, render
    return api, render


@pytest.mark.parametrize("G,Nv", [(1, 1), (5000, 200), (70_001, 300), (100_000, 70_000), (3, 2 ** 20)])
def test_order_is_the_stable_sort_by_nearest_vertex(gpu, G, Nv):
    """One, two and three radix passes (Nv up to 2^8, 2^16, 2^24), ragged
    tile counts, many ties (few vertices)."""
    api, render = gpu
    rng = np.random.default_rng(G + Nv)
    nearest = rng.integers(0, Nv, size=G).astype(np.int32)
    status = api.status_word("cuda")
    got = api.gaussian_order(torch.as_tensor(nearest, device="cuda"), Nv, status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert np.array_equal(got.cpu().numpy(), np.argsort(nearest, kind="stable"))


def test_order_reports_a_bad_index_and_stays_a_permutation(gpu):
    api, render = gpu
    nearest = np.array([3, 9, 1, 3, 0], np.int32)  # 9 is outside [0, 5)
    status = api.status_word("cuda")
    got = api.gaussian_order(torch.as_tensor(nearest, device="cuda"), 5, status).cpu().numpy()
    torch.cuda.synchronize()
    assert int(status.item()) == 7
    assert np.array_equal(np.sort(got), np.arange(5))


@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16, torch.int32])
def test_gather_columns_is_fancy_indexing(gpu, dtype):
    api, render = gpu
    rng = np.random.default_rng(7)
    n = 10_007
    src = torch.as_tensor(rng.normal(size=(4, n)).astype(np.float32) * 1000).to(dtype).cuda()
    order = torch.as_tensor(rng.permutation(n).astype(np.int32), device="cuda")
    status = api.status_word("cuda")
    dst = api.gather_columns(src, order, status)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    assert torch.equal(dst.cpu(), src.cpu()[:, order.cpu().long()])
    bad = order.clone()
    bad[17] = n
    dst = api.gather_columns(src, bad, status)
    torch.cuda.synchronize()
    assert int(status.item()) == 7 and float(dst[:, 17].float().abs().max()) == 0.0


def test_reordered_frame_meets_the_oracle_on_the_reordered_avatar(gpu):
    """The small frame of the avatar stored in nearest-vertex order: the GPU
    order equals numpy's, and every stage meets the oracle run on the same
    reordered avatar (tests/_chain.py, every pixel)."""
    from _chain import chain_check
    api, render = gpu
    sc = scene("c1_small")
    st, order = render.spatially_ordered(render.scene_tensors(sc))
    np_order = synth.nearest_vertex_order(sc)
    assert np.array_equal(order.cpu().numpy(), np_order)
    r = render.Renderer(st)
    torch.cuda.synchronize()
    r.check()
    rep = chain_check(r, synth.permute_gaussians(sc, np_order))
    rep.pop("gpu")
    print("reordered c1_small stage chain:", rep)


@pytest.mark.parametrize("m", [2, 3, 4])
def test_gather_records(gpu, m):
    """Records of m 4-byte words (8, 12, 16 bytes), several rows."""
    api, render = gpu
    rng = np.random.default_rng(m)
    src = torch.as_tensor(rng.normal(size=(3, 513, m)).astype(np.float32), device="cuda")
    order = torch.as_tensor(rng.permutation(513).astype(np.int32), device="cuda")
    dst = api.gather_columns(src, order)
    torch.cuda.synchronize()
    assert torch.equal(dst.cpu(), src.cpu()[:, order.cpu().long(), :])


def test_light_ordered_frame_meets_the_oracle_on_the_reordered_light(gpu):
    """The small frame (8 x 16 light) with its texels in 4 x 8 patches and
    the Gaussians in nearest-vertex order: every stage meets the oracle run
    on the same reordered scene (every pixel), and the image is the one the
    original order renders, up to the summation order of the shading."""
    from _chain import chain_check
    api, render = gpu
    sc = scene("c1_small")
    st0 = render.scene_tensors(sc)
    img0 = render.Renderer(st0).sb.image.clone()
    st, order = render.spatially_ordered(st0)
    lorder = synth.latlong_patch_order(sc.light.rows, sc.light.cols)
    st, _ = render.light_ordered(st, lorder)
    r = render.Renderer(st)
    torch.cuda.synchronize()
    r.check()
    sc2 = synth.permute_lights(synth.permute_gaussians(sc, synth.nearest_vertex_order(sc)), lorder)
    rep = chain_check(r, sc2)
    rep.pop("gpu")
    print("reordered lights and Gaussians, c1_small:", rep)
    assert float((r.sb.image - img0).abs().max()) < 2e-4


@pytest.mark.parametrize("cull_back", [True, False])
def test_faces_ordered_keep_the_bits_and_the_image(gpu, cull_back):
    """Faces stored by normal within each raster chunk: the visibility bits
    (both raster rules, and the paper's triangle-ID form) and the image are
    the original order's bit for bit, and the gathered faces are the
    permuted rows."""
    api, render = gpu
    sc = scene("c1_small")
    st0 = render.scene_tensors(sc)
    forder = synth.face_normal_order(sc.avatar.xv, sc.avatar.faces)
    assert not np.array_equal(forder, np.arange(len(forder)))
    st, o = render.faces_ordered(st0, forder)
    assert np.array_equal(st["avatar"]["faces"].cpu().numpy(), sc.avatar.faces[forder])
    r0 = render.Renderer(st0, vis_cull_back=cull_back)
    r1 = render.Renderer(st, vis_cull_back=cull_back)
    torch.cuda.synchronize()
    r0.check()
    r1.check()
    assert torch.equal(r0.bits, r1.bits)
    assert torch.equal(r0.sb.image, r1.sb.image)
    with pytest.raises(ValueError):
        render.faces_ordered(st0, forder[:-1])


def test_faces_ordered_paper_visibility_keeps_the_counts(gpu):
    api, render = gpu
    sc = scene("c1_small")
    st0 = render.scene_tensors(sc)
    knn_v = torch.as_tensor(np.ascontiguousarray(synth.vertex_knn(sc.avatar.xv, 19).T), dtype=torch.int32,
                            device="cuda")
    st, _ = render.faces_ordered(st0, synth.face_normal_order(sc.avatar.xv, sc.avatar.faces))
    r0 = render.Renderer(st0, visibility="paper", knn_v=knn_v)
    r1 = render.Renderer(st, visibility="paper", knn_v=knn_v)
    torch.cuda.synchronize()
    r0.check()
    r1.check()
    assert torch.equal(r0.vis_count, r1.vis_count)
    assert torch.equal(r0.sb.image, r1.sb.image)
