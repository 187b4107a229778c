"""Stage-by-stage parity of a whole GPU frame with the FP64 oracle.

chain_check(r, sc) takes a Renderer that has just rendered the scene sc and
feeds every oracle stage the GPU's own FP32 outputs of the stage before it,
so each stage is compared on identical inputs:

  skinning    GPU vs the oracle on the avatar rounded to FP32 as the GPU
              holds it (relative to the largest magnitude: 1e-5 for the
              short chains, 5e-5 for normalised vectors and covariances)
  visibility  GPU posed vertices -> orc_visibility (the two-sided rule):
              the light-ordered bits bit for bit, every direction
  shading     GPU skinning outputs + GPU bits -> orc_shade: cull flags bit
              for bit, colours within 2e-4 for every Gaussian
  projection  GPU positions and covariances -> orc_project: means, conics and
              depths relative, rects exactly away from flagged bounds
  binning     GPU rects + depth keys -> orc_bin: the pair count bit for bit,
              each tile list the oracle's in order less pairs whose ellipse
              misses the tile, complete at every checked pixel
  compositing GPU projection + colours -> orc_composite (brute force over
              all Gaussians): colours and final transmittance within 2e-4,
              except the pixels the oracle flags ambiguous, counted

end_to_end_report(r, sc, ref) compares the same frame with the pure oracle
chain (FP64 from the avatar on) and explains every difference above 2e-4:
a Gaussian's colour may differ only where its cull flag or a neighbour's
visibility word differs (FP32 skinning moving a vertex by an ulp across an
integer step), and a pixel only where such a Gaussian reaches it.

Inputs come from the seeded generator; expected values from the oracle only.
"""
import numpy as np

from _common import O, check_tile_lists, f32, light_ordered_bits, rel_err

PIX_TOL = 2e-4


def N(t):
    return t.detach().cpu().numpy()


def gpu_buffers(r):
    """The frame's stage outputs in the oracle's AoS layout."""
    sk = r.sk
    b = r.sb
    P = int(N(b.num_pairs)[0])
    return dict(
        xp=N(sk["xp"]).T, xd=N(sk["xd"]).T, cov=N(sk["cov"]).T, nd=N(sk["nd"]).T, ag=N(sk["ag"]).T,
        rg=N(sk["rg"]).copy(), pg=N(sk["pg"]).copy(), ubar=N(sk["ubar"]).T, bone=N(sk["bone"]).reshape(-1, 3, 4),
        bits=N(r.bits).view(np.uint32), color=N(r.sh["color"]).T, radiance=N(r.sh["radiance"]).T,
        cull=N(r.sh["cull"]), cull_b=N(r.cull_b) if r.overlap else None,
        mean2d=N(b.mean2d).T, conic=N(b.conic).T, depth=N(b.depth).copy(), rect=N(b.rect).T,
        pairs=N(b.pair_gauss)[:P].copy(), tile_range=N(b.tile_range), image=N(b.image).reshape(3, -1).T,
        T_final=N(b.T_final).reshape(-1), tile=b.tile)


def _opacity(sc):
    return f32(sc.avatar.opacity).astype(np.float64)


FLOAT_FIELDS = ("xv", "nv", "wv", "av", "rv", "pv", "dxv", "xg", "logscale", "quat", "opacity", "joints", "pose")


def fp32_avatar(av):
    """The avatar as the GPU holds it: every floating field rounded to FP32
    (and back to FP64 for the oracle).  Identical stage inputs matter in
    Eq. 1: a Gaussian 0.15 mm from a vertex turns the 3e-8 m rounding of its
    position into a 2e-4 relative change of that vertex's distance."""
    import dataclasses
    return dataclasses.replace(av, **{k: f32(getattr(av, k)).astype(np.float64) for k in FLOAT_FIELDS})


def chain_check(r, sc, pixels=None, two_sided=True):
    """Runs every stage comparison (asserting) and returns a report dict.
    sc: the scene as the GPU holds it (BF16-rounded attributes for BF16
    storage); pixels: flat pixel indices for the compositing stage (all
    pixels when None)."""
    g = gpu_buffers(r)
    av = sc.avatar
    rep = {}
    # (a) skinning, on the avatar as the GPU holds it
    av32 = fp32_avatar(av)
    sk = O.skin(av32, O.fk(av32.parents, av32.joints, av32.pose))
    for k, tol in (("xp", 1e-5), ("xd", 1e-5), ("cov", 5e-5), ("nd", 5e-5), ("ag", 1e-5), ("rg", 1e-5),
                   ("pg", 1e-5), ("ubar", 1e-5)):
        e = rel_err(g[k], sk[k])
        rep["skin_" + k] = e
        assert e < tol, f"skinning output {k}: {e:.3g} relative to its largest magnitude (bound {tol})"
    # (b) visibility from the GPU's posed vertices, the oracle's two-sided rule
    xp = f32(g["xp"]).astype(np.float64)
    ref_bits = O.visibility(xp, av.faces, f32(sc.frames.reshape(-1, 9)).astype(np.float64), f32(sc.window_center),
                            float(np.float32(sc.window_half)), float(np.float32(sc.vis_bias)), sc.depth_res,
                            cull_back=not two_sided)
    ref_l = light_ordered_bits(ref_bits, sc.dmap)
    nwords = int((g["bits"] != ref_l).sum())
    rep["visibility_words_differing"] = nwords
    rep["visibility_directions"] = int(sc.frames.shape[0])
    assert nwords == 0, f"{nwords} visibility words differ from the oracle's on the GPU's own posed vertices"
    # (c) shading from the GPU's skinning outputs and bits (light-ordered, so d(k) = k)
    NL = len(sc.light.A)
    ident = np.arange(NL, dtype=np.int32)
    col, rad, cull = O.shade(*(f32(g[k]).astype(np.float64) for k in ("xd", "nd", "ag", "rg", "pg", "ubar")),
                             av.knn, g["bits"], f32(sc.light.L), f32(sc.light.A), f32(sc.light.w), ident,
                             f32(sc.camera.center), g["bits"].shape[1] * 32)
    ncull = int((g["cull"] != cull).sum())
    rep["cull_flags_differing"] = ncull
    assert ncull == 0, f"{ncull} cull flags differ"
    if g["cull_b"] is not None:
        assert np.array_equal(g["cull_b"], cull), "the binning branch's cull flags differ from the shading's"
    keep = cull == 0
    e = float(np.abs(g["color"][keep] - col[keep]).max()) if keep.any() else 0.0
    rep["shade_colour_max_abs"] = e
    rep["shaded_gaussians"] = int(keep.sum())
    assert e < PIX_TOL, f"shading colours: {e:.3g} max-abs (bound {PIX_TOL})"
    assert np.all(g["color"][~keep] == 0.0)
    # L_o relative to its largest value: the GGX peak is the ill-conditioned
    # term - den = (n.h)^2 (alpha^2 - 1) + 1 falls to alpha^2 = gamma^4 >=
    # 0.0081 (roughness >= 0.3), so a few-ulp error in n.h (about 4 x 2^-24)
    # is 2 x 4 x 2^-24 / 0.0081 ~ 6e-5 relative in den and twice that in D
    e = rel_err(g["radiance"][keep], rad[keep]) if keep.any() else 0.0
    rep["shade_radiance_rel"] = e
    assert e < 2e-4, f"shading radiance: {e:.3g} relative to its largest value (bound 2e-4)"
    # (d1) projection from the GPU's skinning outputs and cull flags
    op = _opacity(sc)
    pr = O.project(f32(g["xd"]).astype(np.float64), f32(g["cov"]).astype(np.float64), op, g["cull"], sc.camera)
    valid = pr["valid"] == 1
    for k, tol in (("mean2d", 1e-6), ("conic", 1e-4), ("depth", 1e-6)):
        e = rel_err(g[k][valid], pr[k][valid]) if valid.any() else 0.0
        rep["project_" + k] = e
        assert e < tol, f"projection {k}: {e:.3g} (bound {tol})"
    sure = valid & ~pr["rect_amb"].astype(bool)
    bad = int((g["rect"][sure] != pr["rect"][sure]).any(axis=1).sum())
    rep["rects_flagged"] = int((valid & ~sure).sum())
    assert bad == 0, f"{bad} unflagged rects differ"
    assert np.all(g["rect"][~valid, 2] < g["rect"][~valid, 0]), "an invalid Gaussian has a non-empty rect"
    # (d2, d3) tile lists from the GPU's rects and depth keys: the pair count
    # bit for bit, each list the oracle's in its order less pairs whose
    # ellipse cannot reach the tile, complete at the checked pixels
    W, H = sc.camera.width, sc.camera.height
    start, lst = O.bin_tiles(g["rect"], g["depth"].astype(np.float32).view(np.uint32).copy(), W, H, g["tile"])
    rep["pairs"] = int(len(lst))
    assert len(g["pairs"]) == len(lst), f"{len(g['pairs'])} pairs against the oracle's {len(lst)}"
    kept, _, need = check_tile_lists(g["pairs"], g["tile_range"], start, lst, g["mean2d"], g["conic"],
                                     f32(_opacity(sc)), W, H, g["tile"], pixels)
    rep["pairs_listed"] = kept
    rep["pair_reaches_checked"] = need
    # (d4) compositing from the GPU's projection and colours, brute force
    rgb, T, count, amb = O.composite(f32(g["mean2d"]).astype(np.float64), f32(g["conic"]).astype(np.float64), op,
                                     f32(g["color"]).astype(np.float64), f32(g["depth"]).astype(np.float64),
                                     pr["valid"], W, H, pixels)
    img = g["image"] if pixels is None else g["image"][pixels]
    Tf = g["T_final"] if pixels is None else g["T_final"][pixels]
    ok = amb == 0
    rep["pixels"] = int(len(amb))
    rep["pixels_ambiguous"] = int((~ok).sum())
    e = float(np.abs(img[ok] - rgb[ok]).max()) if ok.any() else 0.0
    rep["pixel_max_abs"] = e
    rep["pixels_covered"] = int((count > 0).sum())
    assert e < PIX_TOL, f"pixels: {e:.3g} max-abs over {int(ok.sum())} unambiguous pixels (bound {PIX_TOL})"
    e = float(np.abs(Tf[ok] - T[ok]).max()) if ok.any() else 0.0
    rep["T_final_max_abs"] = e
    assert e < PIX_TOL
    rep["gpu"] = g
    return rep


def end_to_end_report(g, sc, ref, pixels=None):
    """The GPU frame (buffers g from gpu_buffers) against the pure oracle
    chain ref (oracle.pipeline.frame of the same scene, on the same pixels):
    counts the visibility words and cull flags that differ, and asserts that
    every Gaussian colour and every unambiguous pixel further than 2e-4 from
    the oracle's is touched by one of them."""
    av = sc.avatar
    ref_l = light_ordered_bits(ref["bits"], sc.dmap)
    word_diff = (g["bits"] != ref_l).any(axis=1)              # per vertex
    cull_diff = g["cull"] != ref["cull"]
    touched = cull_diff | word_diff[av.knn].any(axis=1)
    col_bad = np.abs(g["color"] - ref["color"]).max(axis=1) > PIX_TOL
    rep = dict(vertices_with_flipped_bits=int(word_diff.sum()), cull_flips=int(cull_diff.sum()),
               gaussians_touched=int(touched.sum()), gaussian_colours_above_tol=int(col_bad.sum()))
    unexplained = col_bad & ~touched
    assert not unexplained.any(), f"{int(unexplained.sum())} Gaussian colours differ with unchanged inputs"
    img = g["image"] if pixels is None else g["image"][pixels]
    diff = np.abs(img - ref["rgb"]).max(axis=1)
    ok = ref["amb"] == 0
    bad = (diff > PIX_TOL) & ok
    rep["pixels_above_tol"] = int(bad.sum())
    rep["pixel_max_abs_untouched"] = 0.0
    if touched.any() or bad.any():
        # coverage of the touched Gaussians alone: compositing is linear in the
        # colours, so an indicator colour gives > 0 exactly where one of them
        # reaches the pixel with alpha >= 1/255
        sk = ref["skin"]
        pr = O.project(sk["xd"], sk["cov"], av.opacity, None, sc.camera)
        ind = np.repeat(touched.astype(np.float64)[:, None], 3, axis=1)
        W, H = sc.camera.width, sc.camera.height
        cov_rgb, _, _, _ = O.composite(pr["mean2d"], pr["conic"], av.opacity, ind, pr["depth"],
                                       (pr["valid"] & touched).astype(np.int32), W, H, pixels)
        reached = cov_rgb[:, 0] > 0
        unexplained = bad & ~reached
        rep["pixels_reached_by_touched"] = int(reached.sum())
        rep["pixel_max_abs_untouched"] = float(diff[ok & ~reached].max()) if (ok & ~reached).any() else 0.0
        assert not unexplained.any(), f"{int(unexplained.sum())} pixels differ with no touched Gaussian on them"
    else:
        rep["pixel_max_abs_untouched"] = float(diff[ok].max()) if ok.any() else 0.0
    assert rep["pixel_max_abs_untouched"] <= PIX_TOL
    return rep
