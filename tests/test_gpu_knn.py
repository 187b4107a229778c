"""GPU K nearest neighbours (avatar_knn): the sets S_g (K_g nearest vertices of
each Gaussian) and S_v (K_v nearest vertices of each vertex).

The order is defined by the FP64 squared distance (fixed operation order) of
the FP32 coordinates and the index, so the result must equal the oracle's
brute force index for index.
"""
import numpy as np
import pytest

from _common import O, f32, scene, synth

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


def T(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def _knn(api, x, ref, k):
    out = api.avatar_knn(T(f32(x).T), T(f32(ref).T), k)
    torch.cuda.synchronize()
    return out.cpu().numpy().T


@pytest.mark.parametrize("k", [1, 4, 19])
def test_gaussians_to_vertices_and_vertices_to_vertices(gpu, k):
    api = gpu
    av = scene("c1_small").avatar
    got = _knn(api, av.xg, av.xv, k)
    assert np.array_equal(got, O.knn(av.xg, av.xv, k))
    got_v = _knn(api, av.xv, av.xv, k)
    assert np.array_equal(got_v, O.knn(av.xv, av.xv, k))
    assert np.array_equal(got_v[:, 0], np.arange(av.Nv))      # every vertex is its own nearest


def test_paper_scale_on_sampled_queries(gpu):
    api = gpu
    av = scene("c2_paper").avatar
    got = _knn(api, av.xg, av.xv, 3)                           # K_g = 3 as in the paper
    sel = np.random.default_rng(1).choice(av.G, 3000, replace=False)
    assert np.array_equal(got[sel], O.knn(av.xg[sel], av.xv, 3))
    got_v = _knn(api, av.xv, av.xv, 19)                        # K_v = 19
    selv = np.random.default_rng(2).choice(av.Nv, 1000, replace=False)
    assert np.array_equal(got_v[selv], O.knn(av.xv[selv], av.xv, 19))


def test_ties_outside_points_and_degenerate_sets(gpu):
    api = gpu
    rng = np.random.default_rng(4)
    # a lattice: many exact ties, broken by the lower index
    g = np.stack(np.meshgrid(np.arange(6), np.arange(5), np.arange(4), indexing="ij"), -1).reshape(-1, 3) * 0.1
    q = np.concatenate([g + 0.05, rng.uniform(-1, 2, size=(200, 3))])   # centres of cells and points far outside
    assert np.array_equal(_knn(api, q, g, 8), O.knn(q, g, 8))
    # duplicated reference points, K = M, and a single reference point
    ref = np.repeat(rng.normal(size=(10, 3)), 3, axis=0)
    assert np.array_equal(_knn(api, q[:50], ref, 30), O.knn(q[:50], ref, 30))
    assert np.array_equal(_knn(api, q[:50], ref[:1], 1), np.zeros((50, 1), np.int32))
    # a flat (zero-thickness) reference set
    flat = rng.uniform(0, 1, size=(500, 3))
    flat[:, 2] = 0.25
    assert np.array_equal(_knn(api, q, flat, 5), O.knn(q, flat, 5))
    # no query points: nothing to do
    assert api.avatar_knn(T(np.zeros((3, 0), np.float32)), T(f32(g).T), 4).shape == (4, 0)


def test_distances_are_returned(gpu):
    api = gpu
    av = scene("c3_fd").avatar
    d2 = torch.empty(4, av.G, device="cuda")
    idx = api.avatar_knn(T(f32(av.xg).T), T(f32(av.xv).T), 4, dist2=d2)
    torch.cuda.synchronize()
    want_i, want_d = O.knn(av.xg, av.xv, 4, want_dist=True)
    assert np.array_equal(idx.cpu().numpy().T, want_i)
    np.testing.assert_array_equal(d2.cpu().numpy().T, want_d.astype(np.float32))
