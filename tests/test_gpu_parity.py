"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Every test feeds the same seeded inputs to both sides.  Stage tests give
each stage identical FP32 inputs (taken from the oracle's own upstream
stage, rounded to FP32), so integer outputs must match bit for bit and
floating outputs within the stated tolerances:
  visibility bits, tile membership and order : bit-exact
  pixel colours                               : 2e-4 max-abs
  gradients (vs the FP64 adjoint)             : 1e-3 relative per element above 1e-2 of the
                                                group's largest, and 1e-3 |g| + 1e-5 max|g| everywhere
Other FP32 outputs are compared relative to their largest magnitude with
bounds from FP32 rounding (unit roundoff u = 2^-24): a chain of n
operations is within ~n u, so 1e-5 for the short skinning chains, 5e-5 for
normalised vectors, covariances and the 512-term shading sums.
"""
import numpy as np
import pytest

from _common import O, OP, check_tile_lists, f32, light_ordered_bits, oracle_frame, rel_err, scene, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PIX_TOL = 2e-4


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    from paper_2407_10707_gb300 import api, render
    return api, render


def T(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def N(t):
    return t.detach().cpu().numpy()


# ---------------------------------------------------------------- (a) skinning
@pytest.mark.parametrize("name", ["c1_small", "c3_fd"])
def test_skin_matches_oracle(gpu, name):
    api, render = gpu
    sc = scene(name)
    ref = oracle_frame(name)
    st = render.scene_tensors(sc)
    st_status = api.status_word("cuda")
    out = api.avatar_skin(st["avatar"], status=st_status)
    torch.cuda.synchronize()
    api.raise_on_status(st_status)
    sk = ref["skin"]
    assert rel_err(N(out["bone"]).reshape(-1, 3, 4), ref["bone"]) < 1e-5
    assert rel_err(N(out["xp"]).T, sk["xp"]) < 1e-5
    assert rel_err(N(out["xd"]).T, sk["xd"]) < 1e-5
    assert rel_err(N(out["cov"]).T, sk["cov"]) < 5e-5
    assert rel_err(N(out["nd"]).T, sk["nd"]) < 5e-5
    assert rel_err(N(out["ag"]).T, sk["ag"]) < 1e-5
    assert rel_err(N(out["rg"]), sk["rg"]) < 1e-5
    assert rel_err(N(out["pg"]), sk["pg"]) < 1e-5
    assert rel_err(N(out["ubar"]).T, sk["ubar"]) < 1e-5


def test_skin_bad_neighbour_index_sets_status(gpu):
    api, render = gpu
    st = render.scene_tensors(scene("c3_fd"))
    t = dict(st["avatar"])
    knn = t["knn"].clone()
    knn[0, 5] = 10 ** 6
    t["knn"] = knn
    status = api.status_word("cuda")
    api.avatar_skin(t, status=status)
    torch.cuda.synchronize()
    assert int(status.item()) == 7


# ---------------------------------------------------------------- (b) visibility
def _vis_case(sc, xp):
    return dict(xp=T(f32(xp).T), faces=T(sc.avatar.faces, torch.int32), frames=T(f32(sc.frames.reshape(-1, 9))),
                center=sc.window_center, half=sc.window_half, bias=sc.vis_bias, R=sc.depth_res)


def _oracle_bits(sc, xp):
    return O.visibility(f32(xp).astype(np.float64), sc.avatar.faces,
                        f32(sc.frames.reshape(-1, 9)).astype(np.float64), f32(sc.window_center),
                        float(np.float32(sc.window_half)), float(np.float32(sc.vis_bias)), sc.depth_res)


@pytest.mark.parametrize("name,over", [
    ("c1_small", {}),                                             # 64 dirs at 64^2, one CTA per direction
    ("c1_small", dict(n_dirs=128, depth_res=256)),                # 4-CTA clusters
    ("c1_small", dict(n_vertices=10_000, n_dirs=96, depth_res=512)),  # 8-CTA clusters, 1 MB depth maps
    ("c1_small", dict(n_vertices=1_003, n_dirs=32, depth_res=128)),   # ragged vertex count
])
def test_visibility_bits_bit_exact(gpu, name, over):
    api, render = gpu
    sc = synth.config_scene(name, **over)
    sk = O.skin(sc.avatar, O.fk(sc.avatar.parents, sc.avatar.joints, sc.avatar.pose))
    xp = sk["xp"]
    ref = _oracle_bits(sc, xp)
    c = _vis_case(sc, xp)
    status = api.status_word("cuda")
    bits = api.avatar_visibility(c["xp"], c["faces"], c["frames"], c["center"], c["half"], c["bias"], c["R"],
                                 status=status)
    torch.cuda.synchronize()
    api.raise_on_status(status)
    got = N(bits).view(np.uint32)
    assert got.shape == ref.shape
    assert np.array_equal(got, ref), f"{int((got != ref).sum())} words differ"
    # one-sided rasterisation: same bits on this closed mesh, and bit-exact
    # against the oracle's one-sided rule
    ref1 = O.visibility(f32(xp).astype(np.float64), sc.avatar.faces, f32(sc.frames.reshape(-1, 9)).astype(np.float64),
                        f32(sc.window_center), float(np.float32(sc.window_half)), float(np.float32(sc.vis_bias)),
                        sc.depth_res, cull_back=True)
    bits1 = api.avatar_visibility(c["xp"], c["faces"], c["frames"], c["center"], c["half"], c["bias"], c["R"],
                                  cull_back=True)
    torch.cuda.synchronize()
    assert np.array_equal(N(bits1).view(np.uint32), ref1)
    assert np.array_equal(ref1, ref)
    # light-ordered output through d(k)
    dmap = T(sc.dmap, torch.int32)
    bits_l = api.avatar_visibility(c["xp"], c["faces"], c["frames"], c["center"], c["half"], c["bias"], c["R"],
                                   dmap=dmap)
    torch.cuda.synchronize()
    assert np.array_equal(N(bits_l).view(np.uint32), light_ordered_bits(ref, sc.dmap))


@pytest.mark.parametrize("cl", [2, 4, 8])
def test_visibility_cluster_size_knob_keeps_the_bits(gpu, cl):
    """CTAs per direction are a work split only: at 64^2 (one CTA by
    default) and 128^2 the bits at 2, 4 and 8 CTAs per direction are the
    oracle's."""
    api, render = gpu
    from paper_2407_10707_gb300 import _lib as L
    lib = L.load()
    ctx = api.context()
    assert lib.avatar_ctx_set_tuning(ctx, L.TUNE_VIS_CLUSTER, 3) != 0     # not a power of two
    assert lib.avatar_ctx_set_tuning(ctx, L.TUNE_VIS_CLUSTER, 16) != 0    # above the portable cluster size
    try:
        for over in ({}, dict(n_vertices=1_003, n_dirs=32, depth_res=128)):
            sc = synth.config_scene("c1_small", **over)
            sk = O.skin(sc.avatar, O.fk(sc.avatar.parents, sc.avatar.joints, sc.avatar.pose))
            ref = _oracle_bits(sc, sk["xp"])
            c = _vis_case(sc, sk["xp"])
            assert lib.avatar_ctx_set_tuning(ctx, L.TUNE_VIS_CLUSTER, cl) == 0
            assert lib.avatar_ctx_get_tuning(ctx, L.TUNE_VIS_CLUSTER) == cl
            status = api.status_word("cuda")
            bits = api.avatar_visibility(c["xp"], c["faces"], c["frames"], c["center"], c["half"], c["bias"],
                                         c["R"], status=status, cull_back=True)
            torch.cuda.synchronize()
            api.raise_on_status(status)
            assert np.array_equal(N(bits).view(np.uint32), ref)
    finally:
        assert lib.avatar_ctx_set_tuning(ctx, L.TUNE_VIS_CLUSTER, 0) == 0


def test_visibility_edge_cases(gpu):
    api, render = gpu
    rng = np.random.default_rng(3)
    # degenerate triangles, repeated vertices, vertices outside the window, no faces
    xp = rng.uniform(-0.5, 0.5, size=(77, 3))
    xp[5] = [3.0, 0.0, 0.0]                       # outside the window (visible by definition)
    faces = rng.integers(0, 77, size=(150, 3)).astype(np.int32)
    faces[:10, 1] = faces[:10, 0]                 # zero-area triangles
    dirs = synth.fibonacci_directions(64)
    fr = f32(synth.direction_frames(dirs).reshape(-1, 9))
    for F in (150, 0):
        ref = O.visibility(f32(xp).astype(np.float64), faces[:F], fr.astype(np.float64), [0, 0, 0], 1.0, 0.03, 64)
        bits = api.avatar_visibility(T(f32(xp).T), T(faces[:F].reshape(-1, 3), torch.int32), T(fr), [0, 0, 0],
                                     1.0, 0.03, 64)
        torch.cuda.synchronize()
        assert np.array_equal(N(bits).view(np.uint32), ref)
    # argument errors are reported on the host
    with pytest.raises(Exception):
        api.avatar_visibility(T(f32(xp).T), T(faces, torch.int32), T(fr[:30]), [0, 0, 0], 1.0, 0.03, 64)


def test_overlapped_frame_equals_serial_frame(gpu):
    """Projection and binning on a second stream beside visibility and
    shading (avatar_cull's flags, colour records completed by the blend)
    give the serial frame bit for bit, eagerly and from a CUDA graph."""
    api, render = gpu
    st = render.scene_tensors(scene("c1_small"))
    serial = render.Renderer(st, overlap=False)
    img0 = serial.forward().clone()
    torch.cuda.synchronize()
    serial.check()
    r = render.Renderer(st, overlap=True)
    img1 = r.forward().clone()
    torch.cuda.synchronize()
    r.check()
    assert torch.equal(img1, img0)
    assert torch.equal(r.cull_b, serial.sh["cull"])
    assert torch.equal(r.cull_b, r.sh["cull"])
    r.sb.image.zero_()
    r.capture()
    r.replay()
    torch.cuda.synchronize()
    assert torch.equal(r.sb.image, img0)


def test_visibility_wide_chunks_and_bad_index(gpu):
    """Chunks of 1024 triangles whose vertex range exceeds the raster's
    1024-entry vertex cache take the uncached path (the triangles project
    their own vertices); the bits are still the oracle's.  A face with an
    out-of-range index reports AVATAR_ERR_INDEX and its chunk is skipped
    (never read out of bounds)."""
    api, render = gpu
    rng = np.random.default_rng(11)
    nv = 3000
    xp = rng.uniform(-0.6, 0.6, size=(nv, 3))
    # 2,500 triangles: the first two chunks span ~3,000 vertices each (uncached),
    # the ragged third is local (cached)
    far = rng.integers(0, nv, size=(2048, 3))
    near = 100 + rng.integers(0, 40, size=(452, 3))
    faces = np.concatenate([far, near]).astype(np.int32)
    dirs = synth.fibonacci_directions(64)
    fr = f32(synth.direction_frames(dirs).reshape(-1, 9))
    ref = O.visibility(f32(xp).astype(np.float64), faces, fr.astype(np.float64), [0, 0, 0], 1.0, 0.05, 64)
    for cb in (False, True):
        status = api.status_word("cuda")
        bits = api.avatar_visibility(T(f32(xp).T), T(faces, torch.int32), T(fr), [0, 0, 0], 1.0, 0.05, 64,
                                     status=status, cull_back=cb)
        torch.cuda.synchronize()
        api.raise_on_status(status)
        if not cb:
            assert np.array_equal(N(bits).view(np.uint32), ref)
        else:
            ref1 = O.visibility(f32(xp).astype(np.float64), faces, fr.astype(np.float64), [0, 0, 0], 1.0, 0.05, 64,
                                cull_back=True)
            assert np.array_equal(N(bits).view(np.uint32), ref1)
    bad = faces.copy()
    bad[1500, 2] = nv + 5
    status = api.status_word("cuda")
    api.avatar_visibility(T(f32(xp).T), T(bad, torch.int32), T(fr), [0, 0, 0], 1.0, 0.05, 64, status=status,
                          cull_back=True)
    torch.cuda.synchronize()
    assert int(status.item()) == 7


# ---------------------------------------------------------------- (c) shading
@pytest.mark.parametrize("name", ["c1_small", "c3_fd"])
def test_shade_matches_oracle(gpu, name):
    api, render = gpu
    sc = scene(name)
    ref = oracle_frame(name)
    sk = ref["skin"]
    ins = {k: f32(sk[k]) for k in ("xd", "nd", "ag", "rg", "pg", "ubar")}
    cam_c = f32(sc.camera.center)
    light = dict(L=f32(sc.light.L), A=f32(sc.light.A), w=f32(sc.light.w))
    col_ref, rad_ref, cull_ref = O.shade(*(ins[k].astype(np.float64) for k in ("xd", "nd", "ag", "rg", "pg", "ubar")),
                                         sc.avatar.knn, ref["bits"], *(light[k].astype(np.float64) for k in "LAw"),
                                         sc.dmap, cam_c.astype(np.float64), sc.frames.shape[0])
    bits_l = light_ordered_bits(ref["bits"], sc.dmap)
    skt = {k: T(v.T if v.ndim == 2 else v) for k, v in ins.items()}
    lt = {k: T(v) for k, v in light.items()}
    status = api.status_word("cuda")
    out = api.avatar_shade(skt, T(sc.avatar.knn.T, torch.int32), T(bits_l.view(np.int32), torch.int32), lt, cam_c,
                           status=status)
    torch.cuda.synchronize()
    api.raise_on_status(status)
    assert np.array_equal(N(out["cull"]), cull_ref)
    keep = cull_ref == 0
    assert np.abs(N(out["color"]).T[keep] - col_ref[keep]).max() < PIX_TOL
    assert rel_err(N(out["radiance"]).T[keep], rad_ref[keep]) < 5e-5


# ---------------------------------------------------------------- (d) splatting
def _splat_inputs(name):
    sc = scene(name)
    ref = oracle_frame(name)
    sk = ref["skin"]
    return sc, ref, f32(sk["xd"]), f32(sk["cov"]), f32(sc.avatar.opacity), f32(ref["color"]), ref["cull"]


@pytest.mark.parametrize("name", ["c1_small", "c3_fd"])
def test_project_matches_oracle(gpu, name):
    api, render = gpu
    sc, ref, xd, cov, op, col, cull = _splat_inputs(name)
    pr = O.project(xd.astype(np.float64), cov.astype(np.float64), op.astype(np.float64), cull, sc.camera)
    b = api.alloc_splat(xd.shape[0], sc.camera)
    api.avatar_splat_project(T(xd.T), T(cov.T), T(op), T(col.T), T(cull, torch.uint8), sc.camera, b)
    torch.cuda.synchronize()
    valid = pr["valid"] == 1
    assert rel_err(N(b.mean2d).T[valid], pr["mean2d"][valid]) < 1e-6
    assert rel_err(N(b.conic).T[valid], pr["conic"][valid]) < 1e-4
    assert rel_err(N(b.depth)[valid], pr["depth"][valid]) < 1e-6
    rect = N(b.rect).T
    sure = ~pr["rect_amb"].astype(bool)
    assert np.array_equal(rect[sure], pr["rect"][sure])
    assert sure.mean() > 0.97   # four bounds, each within 2e-3 px of an integer with p ~ 4e-3


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_bin_tile_lists_against_oracle(gpu, tile):
    """The pair count bit for bit; each tile list the oracle's rect list of
    that tile in its (depth, index) order less pairs whose ellipse cannot
    reach the tile, and complete at every pixel (tests/_common.py)."""
    api, render = gpu
    sc, ref, xd, cov, op, col, cull = _splat_inputs("c1_small")
    pr = O.project(xd.astype(np.float64), cov.astype(np.float64), op.astype(np.float64), cull, sc.camera)
    depth32 = f32(pr["depth"])
    key = depth32.view(np.uint32).copy()
    start, lst = O.bin_tiles(pr["rect"], key, sc.camera.width, sc.camera.height, tile)
    G = xd.shape[0]
    b = api.alloc_splat(G, sc.camera, tile=tile)
    b.rect.copy_(T(pr["rect"].T, torch.int32))
    b.depth.copy_(T(depth32))
    b.mean2d.copy_(T(f32(pr["mean2d"]).T))
    b.conic.copy_(T(f32(pr["conic"]).T))
    status = api.status_word("cuda")
    api.avatar_splat_bin(T(xd.T), T(cov.T), T(op), T(col.T), T(cull, torch.uint8), sc.camera, b, status=status)
    torch.cuda.synchronize()
    api.raise_on_status(status)
    P = int(N(b.num_pairs)[0])
    assert P == len(lst)
    kept, total, need = check_tile_lists(N(b.pair_gauss)[:P], N(b.tile_range), start, lst, f32(pr["mean2d"]),
                                         f32(pr["conic"]), op.astype(np.float32), sc.camera.width,
                                         sc.camera.height, tile)
    print(f"tile {tile}: {kept} of {total} pairs listed, {need} (pixel, Gaussian) reaches checked")
    assert 0 < kept <= total and need > 0


@pytest.mark.parametrize("name,tile,ppt", [("c1_small", 16, 1), ("c3_fd", 8, 1), ("c1_small", 32, 1),
                                           ("c1_small", 16, 2), ("c1_small", 16, 4), ("c3_fd", 8, 2),
                                           ("c1_small", 32, 2), ("c1_small", 32, 4)])
def test_blend_matches_bruteforce_oracle(gpu, name, tile, ppt):
    """The blend at every tile edge and pixels-per-thread split (each warp
    item a box of 8 x 4 ppt pixels) against brute-force compositing."""
    api, render = gpu
    from paper_2407_10707_gb300 import _lib as L
    lib = L.load()
    assert lib.avatar_ctx_set_tuning(api.context(), L.TUNE_BLEND_PPT, ppt) == 0
    try:
        _blend_case(api, name, tile)
    finally:
        assert lib.avatar_ctx_set_tuning(api.context(), L.TUNE_BLEND_PPT, 1) == 0


def _elongated_cov(G, seed=5, scales=(0.12, 2e-4, 2e-4)):
    """Covariances R diag(s^2) R^T of random rotations with one axis 600x
    the others (projected: ellipses up to 180 pixels long, det / (a c) of
    the conic down to 1e-3), in the [G][6] (xx, xy, xz, yy, yz, zz) layout."""
    rng = np.random.default_rng(seed)
    q = rng.normal(size=(G, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    R = np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                  2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                  2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], 1).reshape(G, 3, 3)
    s = np.asarray(scales)[None] * rng.uniform(0.5, 2.0, size=(G, 3))
    S = np.einsum("gij,gj,gkj->gik", R, s * s, R)
    return f32(np.stack([S[:, 0, 0], S[:, 0, 1], S[:, 0, 2], S[:, 1, 1], S[:, 1, 2], S[:, 2, 2]], 1))


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_blend_of_elongated_gaussians_matches_bruteforce_oracle(gpu, tile):
    """Thin, long, rotated ellipses spanning up to six 32-pixel tiles: the
    tile lists and region masks drop only pairs whose ellipse cannot reach a
    pixel (the reach tests run on conics near their degenerate limit), so the
    image meets brute-force compositing as everywhere else."""
    api, render = gpu
    sc = scene("c1_small")
    _blend_case(api, "c1_small", tile, cov=_elongated_cov(sc.avatar.G))


def _blend_case(api, name, tile, cov=None):
    sc, ref, xd, cov0, op, col, cull = _splat_inputs(name)
    cov = cov0 if cov is None else cov
    pr = O.project(xd.astype(np.float64), cov.astype(np.float64), op.astype(np.float64), cull, sc.camera)
    m32, c32, d32 = f32(pr["mean2d"]), f32(pr["conic"]), f32(pr["depth"])
    W, H = sc.camera.width, sc.camera.height
    rgb, Tf, cnt, amb = O.composite(m32.astype(np.float64), c32.astype(np.float64), op.astype(np.float64),
                                    col.astype(np.float64), d32.astype(np.float64), pr["valid"], W, H)
    G = xd.shape[0]
    b = api.alloc_splat(G, sc.camera, tile=tile)
    b.rect.copy_(T(pr["rect"].T, torch.int32))
    b.depth.copy_(T(d32))
    b.mean2d.copy_(T(m32.T))
    b.conic.copy_(T(c32.T))
    args = (T(xd.T), T(cov.T), T(op), T(col.T), T(cull, torch.uint8), sc.camera, b)
    api.avatar_splat_bin(*args)
    api.avatar_splat_blend(*args)
    torch.cuda.synchronize()
    img = N(b.image).reshape(3, -1).T
    ok = amb == 0
    assert ok.mean() > 0.99
    err = np.abs(img[ok] - rgb[ok]).max()
    assert err < PIX_TOL, err
    assert np.abs(N(b.T_final).reshape(-1)[ok] - Tf[ok]).max() < PIX_TOL


def test_image_is_tile_size_invariant_and_graph_replay_is_identical(gpu):
    api, render = gpu
    st = render.scene_tensors(scene("c1_small"))
    imgs = []
    for tile in (8, 16, 32):
        r = render.Renderer(st, tile=tile)
        imgs.append(N(r.forward()).copy())
        r.check()
    assert np.array_equal(imgs[0], imgs[1]) and np.array_equal(imgs[1], imgs[2])
    r = render.Renderer(st)
    eager = N(r.forward()).copy()
    r.capture()
    r.replay()
    torch.cuda.synchronize()
    assert np.array_equal(N(r.sb.image), eager)


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_region_masks_change_neither_image_nor_gradients(gpu, tile):
    """Pair keys carry the mask of the tile regions a Gaussian's ellipse
    reaches and the blends skip the boxes it misses; with the masks off
    (AVATAR_TUNE_REGION_MASKS = 0, the form past 2^24 tiles) the blends use
    the rect test alone.  Both must give the same image bit for bit (the
    skipped hits add nothing) and the same gradients up to the order of the
    atomic additions."""
    api, render = gpu
    from paper_2407_10707_gb300 import _lib as L
    lib, ctx = L.load(), api.context()
    st = render.scene_tensors(scene("c1_small"))
    target = torch.as_tensor(np.full((3, 256, 256), 0.3, np.float32), device="cuda")
    out = {}
    try:
        for masks in (1, 0):
            assert lib.avatar_ctx_set_tuning(ctx, L.TUNE_REGION_MASKS, masks) == 0
            ts = render.TrainStep(st, target, tile=tile)
            torch.cuda.synchronize()
            ts.check()
            out[masks] = (N(ts.sb.image).copy(), {k: N(v).copy() for k, v in ts.grads().items()},
                          int(N(ts.sb.num_pairs)[0]))
    finally:
        lib.avatar_ctx_set_tuning(ctx, L.TUNE_REGION_MASKS, 1)
    assert lib.avatar_ctx_set_tuning(ctx, L.TUNE_REGION_MASKS, 2) != 0
    assert out[1][2] == out[0][2]                       # the same pairs are emitted either way
    assert np.array_equal(out[1][0], out[0][0])
    for k in out[1][1]:
        assert rel_err(out[1][1][k], out[0][1][k]) < 1e-5, k


def test_pair_overflow_is_reported_not_faulted(gpu):
    api, render = gpu
    st = render.scene_tensors(scene("c3_fd"))
    r = render.Renderer(st, pair_capacity=64)
    torch.cuda.synchronize()
    assert int(r.status.item()) == 3
    assert int(N(r.sb.num_pairs)[0]) > 64
    assert float(N(r.sb.image).max()) == 0.0


def test_sort_wait_that_runs_out_reports_timeout_and_keeps_the_image(gpu):
    """The radix sorts of splatting with one poll allowed per look-back wait
    (AVATAR_TUNE_WAIT_LIMIT = 1) on the paper-scale frame (98 depth-sort
    tiles, ~1,000 tile-sort tiles): some block finds a predecessor not yet
    published and gives up, the status word reads AVATAR_ERR_TIMEOUT, the
    call returns, and the expired blocks' exact fallback leaves the image
    bit for bit the default one."""
    api, render = gpu
    from paper_2407_10707_gb300 import _lib as L
    lib = L.load()
    ctx = api.context()
    assert lib.avatar_ctx_set_tuning(ctx, L.TUNE_WAIT_LIMIT, -1) != 0
    st = render.scene_tensors(scene("c2_paper"))
    r = render.Renderer(st)
    torch.cuda.synchronize()
    r.check()
    img0 = r.sb.image.clone()
    assert lib.avatar_ctx_set_tuning(ctx, L.TUNE_WAIT_LIMIT, 1) == 0
    try:
        seen = []
        for _ in range(5):           # expiry depends on block timing; one poll makes it near certain
            r.status.zero_()
            r.sb.image.zero_()
            r.forward()
            torch.cuda.synchronize()
            seen.append(int(r.status.item()))
            assert seen[-1] in (0, 4), seen
            assert torch.equal(r.sb.image, img0)
            if seen[-1] == 4:
                break
        print(f"status per attempt with one poll per wait: {seen}")
        assert seen[-1] == 4, f"no wait ran out in {len(seen)} frames"
    finally:
        assert lib.avatar_ctx_set_tuning(ctx, L.TUNE_WAIT_LIMIT, 0) == 0
    r.status.zero_()
    r.forward()
    torch.cuda.synchronize()
    r.check()
    assert torch.equal(r.sb.image, img0)


# ---------------------------------------------------------------- whole frame
@pytest.mark.parametrize("name", ["c1_small", "c3_fd"])
def test_frame_end_to_end(gpu, name):
    """The whole frame, stage by stage on the GPU's own inputs (every pixel),
    then against the pure oracle chain with every difference above 2e-4
    explained by a flipped visibility bit or cull flag (tests/_chain.py)."""
    from _chain import chain_check, end_to_end_report
    api, render = gpu
    sc = scene(name)
    st = render.scene_tensors(sc)
    r = render.Renderer(st)
    r.forward()
    torch.cuda.synchronize()
    r.check()
    rep = chain_check(r, sc)
    g = rep.pop("gpu")
    print(f"{name} stage chain:", rep)
    e2e = end_to_end_report(g, sc, oracle_frame(name))
    print(f"{name} end to end:", e2e)


# ---------------------------------------------------------------- gradients
def _fd_problem(gpu):
    api, render = gpu
    from oracle import adjoint as AJ
    sc = scene("c3_fd")
    ref = oracle_frame("c3_fd")
    av = sc.avatar
    rng = np.random.default_rng(5)
    target = np.clip(ref["rgb"] * rng.uniform(0.8, 1.2, ref["rgb"].shape), 0, None)
    fixed = dict(knn=av.knn, xv=AJ.t64(av.xv), dxv=AJ.t64(av.dxv), nv=AJ.t64(av.nv), bone=AJ.t64(ref["bone"]),
                 bits=ref["bits"], dmap=sc.dmap, A=AJ.t64(sc.light.A), w=AJ.t64(sc.light.w),
                 cam_center=AJ.t64(sc.camera.center), culled=ref["cull"], valid=ref["proj"]["valid"], cam=sc.camera)
    params = dict(xg=av.xg, logscale=av.logscale, quat=av.quat, opacity=av.opacity, av=av.av, rv=av.rv, pv=av.pv,
                  L=sc.light.L, wv=av.wv)
    tp = {k: AJ.t64(v).requires_grad_(True) for k, v in params.items()}
    img = AJ.render(tp, fixed)
    loss = AJ.l1_loss(img, AJ.t64(target).reshape(img.shape))
    loss.backward()
    return sc, ref, target, {k: v.grad.numpy() for k, v in tp.items()}, float(loss)


@pytest.fixture(scope="module")
def fd_problem(gpu):
    return _fd_problem(gpu)


@pytest.mark.parametrize("bppt", [1, 2, 4])
def test_train_step_gradients_match_fp64_adjoint(gpu, fd_problem, bppt):
    """Train-step gradients of every trainable group against the FP64
    adjoint (which the oracle pins check against central finite
    differences), element by element, at each pixels-per-thread split of the
    compositing adjoint."""
    api, render = gpu
    from paper_2407_10707_gb300 import _lib as L
    lib = L.load()
    assert lib.avatar_ctx_set_tuning(api.context(), L.TUNE_BLEND_BWD_PPT, bppt) == 0
    try:
        _grad_case(gpu, fd_problem, bppt)
    finally:
        assert lib.avatar_ctx_set_tuning(api.context(), L.TUNE_BLEND_BWD_PPT, 1) == 0


def _grad_case(gpu, fd_problem, bppt):
    api, render = gpu
    sc, ref, target, g_ref, loss_ref = fd_problem
    st = render.scene_tensors(sc)
    W, H = sc.camera.width, sc.camera.height
    tgt = T(f32(target).T.reshape(3, H, W))
    ts = render.TrainStep(st, tgt, ssim_weight=0.0)
    loss = float(ts.step().item())
    torch.cuda.synchronize()
    ts.check()
    assert abs(loss - loss_ref) < 1e-3 * abs(loss_ref) + 1e-6
    g = {k: N(v) for k, v in ts.grads().items()}
    pairs = dict(xg=(g["xg"].T, g_ref["xg"]), logscale=(g["logscale"].T, g_ref["logscale"]),
                 quat=(g["quat"].T, g_ref["quat"]), opacity=(g["opacity"], g_ref["opacity"]),
                 av=(g["av"].T, g_ref["av"]), rv=(g["rv"], g_ref["rv"]), pv=(g["pv"], g_ref["pv"]),
                 L=(g["L"], g_ref["L"]), wv=(g["wv"], g_ref["wv"]))
    worst = {}
    for k, (got, want) in pairs.items():
        worst[k] = grad_agreement(got, want, k)
    print(f"backward pixels/thread {bppt}: per-element relative error (|g| > 1e-2 max), max-normalised error, "
          f"elements in (1e-3, 1e-2] x max beyond 1e-3 relative:",
          {k: (f"{a:.2e}", f"{b:.2e}", c) for k, (a, b, c) in worst.items()})


def grad_agreement(got, ref, name, rtol=1e-3, floor=1e-2, atol_frac=1e-5):
    """Per-element gradient check: every element whose reference magnitude
    exceeds floor x the group's largest is within rtol relative, and every
    element within rtol |ref| + atol_frac x the largest.  The absolute
    floor covers FP32 cancellation: an element is a sum of terms of both
    signs (pixels' residual signs, colour channels, lights), each evaluated
    to ~2^-24 of its own size, so an element that cancels to a small share
    of its terms keeps their absolute error.  On the 1,000-Gaussian problem
    one roughness element at 1.1e-3 of its group's largest comes from one
    Gaussian whose three colour-channel terms cancel about 100-fold, and is
    2e-3 off relative (1.6e-11 absolute, 2e-6 of the largest).  The count of
    elements between 1e-3 and floor x the largest that miss rtol is
    returned too.  Returns (worst per-element relative error over the first
    set, max error / largest, misses in the band)."""
    got = np.asarray(got, np.float64).reshape(-1)
    ref = np.asarray(ref, np.float64).reshape(-1)
    m = float(np.abs(ref).max())
    if m == 0.0:
        assert np.all(got == 0.0), name
        return 0.0, 0.0, 0
    band = (np.abs(ref) > 1e-3 * m) & (np.abs(ref) <= floor * m)
    band_miss = int((np.abs(got[band] - ref[band]) > rtol * np.abs(ref[band])).sum())
    big = np.abs(ref) > floor * m
    rel = np.abs(got[big] - ref[big]) / np.abs(ref[big])
    worst = float(rel.max()) if big.any() else 0.0
    i = int(np.argmax(rel)) if big.any() else 0
    assert worst <= rtol, (f"{name}: element {int(np.flatnonzero(big)[i])} off by {worst:.3g} relative "
                           f"({got[big][i]:.6g} vs {ref[big][i]:.6g})")
    over = np.abs(got - ref) > rtol * np.abs(ref) + atol_frac * m
    if over.any():
        j = int(np.argmax(np.where(over, np.abs(got - ref), 0.0)))
        raise AssertionError(f"{name}: {int(over.sum())} small elements beyond rtol |ref| + {atol_frac} max|ref|; "
                             f"worst {got[j]:.6g} vs {ref[j]:.6g} (max|ref| {m:.6g})")
    return worst, float(np.abs(got - ref).max() / m), band_miss


def test_autograd_wrappers_match_train_step(gpu):
    api, render = gpu
    sc = scene("c3_fd")
    ref = oracle_frame("c3_fd")
    st = render.scene_tensors(sc)
    t = st["avatar"]
    r = render.Renderer(st)
    bits = r.bits.clone()
    params = {k: t[k].clone().requires_grad_(True) for k in ("xg", "logscale", "quat", "opacity", "wv", "av", "rv",
                                                               "pv")}
    params["L"] = st["light"]["L"].clone().requires_grad_(True)
    img = render.render_differentiable(params, st, bits)
    tgt = torch.zeros_like(img)
    loss = render.L1Fn.apply(img, tgt)
    loss.backward()
    ts = render.TrainStep(st, tgt, ssim_weight=0.0)
    ts.step()
    torch.cuda.synchronize()
    g = ts.grads()
    for k in ("xg", "logscale", "quat", "opacity", "wv", "av", "rv", "pv", "L"):
        assert rel_err(N(params[k].grad), N(g[k])) < 1e-4, k
    np.testing.assert_allclose(float(loss), float(ts.loss.item()), rtol=1e-6)
