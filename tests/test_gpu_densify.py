"""The density-based densification of App. B / Alg. 1 on the GPU
(avatar_densify) against the oracle: the vertex counts D_v, the number of
added Gaussians N', each draw's triangle and the per-triangle counts are
bit-exact (integer decisions throughout); the FP32 positions are within
8 FP32 steps of the coordinates' magnitude (two differences, two products,
two sums)."""
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


def _words(n, seed):
    return np.random.default_rng(seed).integers(0, 2 ** 32, size=(3, n), dtype=np.uint64).astype(np.uint32)


def _run(api, knn, faces, xv, words, d0=1.0, p0=0.02, status=None):
    dev = "cuda"
    out = api.avatar_densify(torch.as_tensor(np.ascontiguousarray(knn.T), dtype=torch.int32, device=dev),
                             torch.as_tensor(np.ascontiguousarray(faces), dtype=torch.int32, device=dev),
                             torch.as_tensor(np.ascontiguousarray(xv.T), dtype=torch.float32, device=dev),
                             torch.as_tensor(words.view(np.int32), device=dev), d0, p0, status=status,
                             want_stats=True)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _check(got, knn, faces, xv, words, d0=1.0, p0=0.02):
    """words: the uniform words the oracle draws from (at least as many as
    the kernel's capacity; the kernel used the first capacity columns)."""
    from oracle import densify as DN
    xv32 = np.asarray(xv, np.float32).astype(np.float64)
    cap = got["tri"].shape[0]
    want = DN.densify(knn, faces, xv32, words.T.astype(np.uint64), d0, p0)
    np.testing.assert_array_equal(got["Dv"], want["Dv"])
    np.testing.assert_array_equal(got["df"], want["df"].astype(np.float32))
    assert int(got["count"][0]) == want["n_new"]
    n = min(want["n_new"], cap)
    np.testing.assert_array_equal(got["tri"][:n], want["tri"][:n])
    np.testing.assert_array_equal(got["ng"], np.bincount(want["tri"][:n], minlength=len(faces)))
    scale = np.abs(xv32).max()
    assert np.abs(got["x"][:, :n].T - want["x"][:n]).max() <= 8 * 2.0 ** -24 * scale
    return want


def test_densify_matches_oracle_small(gpu):
    sc = scene("c1_small")
    av = sc.avatar
    # thin the Gaussians so that many triangles are under-covered
    keep = np.random.default_rng(1).choice(av.knn.shape[0], 1500, replace=False)
    knn = av.knn[keep][:, :3]
    words = _words(4000, 2)
    got = _run(gpu, knn, av.faces, av.xv, words)
    want = _check(got, knn, av.faces, av.xv, words)
    assert want["n_new"] > 10


def test_densify_matches_oracle_paper_scale(gpu):
    """The 50k-vertex, 100k-triangle mesh with every eighth of its 200k
    Gaussians (K_g = 3), so that most triangles are under-covered; p0 = 0.02
    and 0.2 (about 1.5k and 15k draws)."""
    sc = scene("c2_paper")
    av = sc.avatar
    knn = av.knn[::8, :3]
    words = _words(20000, 3)
    for p0 in (0.02, 0.2):
        got = _run(gpu, knn, av.faces, av.xv, words, p0=p0)
        _check(got, knn, av.faces, av.xv, words, p0=p0)


def test_densify_edge_cases(gpu):
    api = gpu
    sc = scene("c1_small")
    av = sc.avatar
    F = len(av.faces)
    # no Gaussians: every triangle has density 0, N' = floor(0.02 F)
    words = _words(200, 4)
    got = _run(api, np.zeros((0, 3), np.int64), av.faces, av.xv, words)
    _check(got, np.zeros((0, 3), np.int64), av.faces, av.xv, words)
    assert int(got["count"][0]) == int(np.floor(0.02 * F))
    # saturated: every vertex in S_g of many Gaussians, nothing added
    knn = np.repeat(np.arange(av.xv.shape[0]), 4)[:, None].repeat(3, 1)
    got = _run(api, knn, av.faces, av.xv, _words(10, 5))
    assert int(got["count"][0]) == 0 and got["ng"].sum() == 0
    # capacity below N': the first capacity draws, N' reported, overflow flagged
    st = api.status_word("cuda")
    words = _words(200, 6)
    got = _run(api, np.zeros((0, 3), np.int64), av.faces, av.xv, words[:, :7].copy(), status=st)
    assert int(st.item()) == 3  # AVATAR_ERR_OVERFLOW
    want = _check(got, np.zeros((0, 3), np.int64), av.faces, av.xv, words)
    assert want["n_new"] > 7
    # a bad neighbour index is reported and skipped
    st = api.status_word("cuda")
    bad = av.knn[:100, :3].copy()
    bad[5, 1] = av.xv.shape[0] + 3
    _run(api, bad, av.faces, av.xv, _words(100, 7), status=st)
    assert int(st.item()) != 0


def test_densify_grows_the_avatar(gpu):
    api = gpu
    from paper_2407_10707_gb300 import render
    sc = scene("c1_small")
    st = render.scene_tensors(sc, "cuda")
    t = st["avatar"]
    G0 = t["xg"].shape[1]
    keep = torch.arange(0, G0, 8, device="cuda")
    for k in ("xg", "logscale", "quat"):
        t[k] = t[k][:, keep].contiguous()
    t["opacity"] = t["opacity"][keep].contiguous()
    t["knn"] = t["knn"][:, keep].contiguous()
    g1 = t["xg"].shape[1]
    words = torch.as_tensor(_words(5000, 9).view(np.int32), device="cuda")
    n = render.densify(st, words)
    assert n > 0 and t["xg"].shape[1] == g1 + n and t["knn"].shape[1] == g1 + n
    # the new neighbour lists are the exact K nearest vertices of every Gaussian
    from oracle import oracle as O
    want = O.knn(t["xg"].cpu().numpy().T, t["xv"].cpu().numpy().T, t["knn"].shape[0])
    np.testing.assert_array_equal(t["knn"].cpu().numpy().T, want)
    r = render.Renderer(st)
    r.forward()
    r.check()


def test_densify_zero_capacity_reports_the_count(gpu):
    api = gpu
    sc = scene("c1_small")
    av = sc.avatar
    st = api.status_word("cuda")
    words = _words(0, 1).reshape(3, 0)
    got = _run(api, np.zeros((0, 3), np.int64), av.faces, av.xv, words, status=st)
    assert int(got["count"][0]) == int(np.floor(0.02 * len(av.faces)))
    assert int(st.item()) == 3 and got["ng"].sum() == 0  # overflow flagged, nothing drawn
