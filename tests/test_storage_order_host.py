"""Host-side storage orders of the input generator (no GPU): the light
texels' patch order and the Gaussians' nearest-vertex order are
permutations with the stated structure, and permuting a scene moves every
per-Gaussian / per-texel field together."""
import numpy as np

from paper_2407_10707_gb300 import synth


def test_patch_order_is_a_permutation_of_4x8_blocks():
    o = synth.latlong_patch_order(16, 32)
    assert np.array_equal(np.sort(o), np.arange(512))
    for p in range(16):
        blk = o[32 * p:32 * p + 32]
        rows, cols = blk // 32, blk % 32
        assert len(np.unique(rows)) == 4 and len(np.unique(cols)) == 8
        assert rows.max() - rows.min() == 3 and cols.max() - cols.min() == 7
    assert np.array_equal(synth.latlong_patch_order(6, 10), np.arange(60))   # no 4 x 8 split: identity


def test_nearest_vertex_order_and_scene_permutations():
    sc = synth.config_scene("c3_fd")
    o = synth.nearest_vertex_order(sc)
    assert np.array_equal(np.sort(o), np.arange(sc.avatar.G))
    k0 = sc.avatar.knn[o, 0]
    assert np.all(np.diff(k0) >= 0)
    ties = np.diff(k0) == 0
    assert np.all(np.diff(o)[ties] > 0)                      # stable: ties keep the original order
    sp = synth.permute_gaussians(sc, o)
    for f in ("xg", "logscale", "quat", "opacity", "knn"):
        assert np.array_equal(getattr(sp.avatar, f), getattr(sc.avatar, f)[o])
    assert np.array_equal(sp.avatar.xv, sc.avatar.xv)
    lo = synth.latlong_patch_order(8, 16)
    sl = synth.permute_lights(sc, lo)
    assert np.array_equal(sl.light.L, sc.light.L[lo]) and np.array_equal(sl.light.w, sc.light.w[lo])
    assert np.array_equal(sl.light.A, sc.light.A[lo]) and np.array_equal(sl.dmap, np.asarray(sc.dmap)[lo])
