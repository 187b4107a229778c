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


def test_face_normal_order_permutes_within_raster_chunks():
    """The faces' storage order keeps every raster chunk's faces (so each
    chunk's vertex range) and lists them by octahedral normal bin, stably;
    the chunk is the library's."""
    from paper_2407_10707_gb300 import _lib as L
    sc = synth.config_scene("c1_small")
    xv, faces = sc.avatar.xv, sc.avatar.faces
    o = synth.face_normal_order(xv, faces, chunk=L.VIS_FACE_CHUNK)
    F = len(faces)
    assert np.array_equal(np.sort(o), np.arange(F))
    for c in range(0, F, L.VIS_FACE_CHUNK):
        blk = o[c:c + L.VIS_FACE_CHUNK]
        assert blk.min() >= c and blk.max() < min(F, c + L.VIS_FACE_CHUNK)
    # faces of a sphere in random order: listed by normal bin, neighbours in
    # the order face nearly the same way
    v, f, _ = synth._tessellate_capsule((0, 0, 0), (0, 0, 0), 0.5, 600)
    f = f[np.random.default_rng(3).permutation(len(f))]
    o2 = synth.face_normal_order(v, f, chunk=L.VIS_FACE_CHUNK)
    n = np.cross(v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    step = lambda nn: float(np.mean(np.sum(nn[1:] * nn[:-1], axis=1)))   # mean cosine of consecutive normals
    assert step(n) < 0.1 and step(n[o2]) > 0.7
    sp = synth.permute_faces(sc, o)
    assert np.array_equal(sp.avatar.faces, faces[o])


def test_hilbert_index_walks_neighbouring_cells():
    """The face order's curve: on an 8 x 8 grid the index is a bijection
    onto 0..63 and consecutive indices are edge-adjacent cells."""
    n = 8
    x, y = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    d = synth._hilbert_index(x.ravel(), y.ravel(), n)
    assert np.array_equal(np.sort(d), np.arange(n * n))
    pos = np.empty((n * n, 2), np.int64)
    pos[d] = np.c_[x.ravel(), y.ravel()]
    assert np.all(np.abs(np.diff(pos, axis=0)).sum(axis=1) == 1)
