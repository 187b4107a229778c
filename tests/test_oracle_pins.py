"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: closed
forms, invariants, special cases, constants printed in the paper
(tests/golden/), an independent restatement, or central finite differences.
No GPU is used.
"""
import copy
import math
import os

import numpy as np
import pytest
import torch

from oracle import adjoint as AJ
from oracle import oracle as O
from oracle import pipeline as OP
from paper_2407_10707_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden_constants(name="app_a_brdf_constants.txt"):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split()[:2]
                vals[k] = float(v)
    return vals


def rot(axis, ang):
    axis = np.asarray(axis, float)
    axis = axis / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * K @ K


@pytest.fixture(scope="module")
def small_avatar():
    return synth.make_avatar(642, 300, seed=5)


# ---------------------------------------------------------------- FK / skin
def test_fk_identity_pose_gives_identity_bones():
    pose = np.zeros((24, 3))
    bone = O.fk(synth.PARENTS, synth.REST_JOINTS, pose)
    for j in range(24):
        np.testing.assert_allclose(bone[j, :, :3], np.eye(3), atol=1e-15)
        np.testing.assert_allclose(bone[j, :, 3], 0, atol=1e-15)


def test_fk_root_rotation_is_rigid():
    pose = np.zeros((24, 3))
    pose[0] = [0.2, -0.4, 0.3]
    Q = rot(pose[0], np.linalg.norm(pose[0]))
    J0 = synth.REST_JOINTS[0]
    bone = O.fk(synth.PARENTS, synth.REST_JOINTS, pose)
    for j in range(24):
        np.testing.assert_allclose(bone[j, :, :3], Q, atol=1e-13)
        np.testing.assert_allclose(bone[j, :, 3], J0 - Q @ J0, atol=1e-13)


def test_fk_chain_closed_form():
    parents = np.array([-1, 0, 1], np.int32)
    joints = np.array([[0.0, 0, 0], [1.0, 0, 0], [2.0, 0, 0]])
    pose = np.array([[0, 0, math.pi / 2], [0, 0, math.pi / 2], [0, 0, 0]])
    bone = O.fk(parents, joints, pose)
    # joint 1 moves to R0 (J1 - J0) = (0,1,0); joint 2 to (0,1,0) + R0 R1 (1,0,0) = (-1,1,0)
    apply = lambda j, x: bone[j, :, :3] @ x + bone[j, :, 3]
    np.testing.assert_allclose(apply(1, joints[1]), [0, 1, 0], atol=1e-14)
    np.testing.assert_allclose(apply(2, joints[2]), [-1, 1, 0], atol=1e-14)


def test_fk_chain_noncommuting_rotations():
    """The parent's rotation acts after the child's (T_j = T_parent [R_j | J_j - J_parent]):
    joint 0 turns 90 degrees about x, joint 1 (rest (1,0,0)) 90 degrees about z.
    A point at (2,0,0) bound to joint 1 goes to J0 + R0 (R1 (x - J1) + (J1 - J0))
    = R0 ((0,1,0) + (1,0,0)) = (1,0,1); the reversed product R1 R0 would give (1,1,0)."""
    parents = np.array([-1, 0], np.int32)
    joints = np.array([[0.0, 0, 0], [1.0, 0, 0]])
    pose = np.array([[math.pi / 2, 0, 0], [0, 0, math.pi / 2]])
    bone = O.fk(parents, joints, pose)
    x = np.array([2.0, 0.0, 0.0])
    np.testing.assert_allclose(bone[1, :, :3] @ x + bone[1, :, 3], [1, 0, 1], atol=1e-14)
    np.testing.assert_allclose(bone[1, :, :3], rot([1, 0, 0], math.pi / 2) @ rot([0, 0, 1], math.pi / 2),
                               atol=1e-14)


def test_skin_eq1_inverse_distance_weights(small_avatar):
    """Eq. 1: u_j = 1 / |x_g - x_j| over S_g, normalised.  Gaussian 0's four
    neighbours are moved to distances 1, 2, 4 and 4 cm from it (in different
    directions): ubar = (1, 1/2, 1/4, 1/4) / 2, and each interpolated
    attribute is that mix of the neighbours' values (identity pose)."""
    av = copy.deepcopy(small_avatar)
    av.pose = np.zeros((24, 3))
    nb = av.knn[0]
    assert av.K == 4 and len(set(nb.tolist())) == 4
    dirs = np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0], [-1.0, 0, 0]])
    for j, d in enumerate((1.0, 2.0, 4.0, 4.0)):
        av.xv[nb[j]] = av.xg[0] + 0.01 * d * dirs[j]
    sk = O.skin(av, O.fk(av.parents, av.joints, av.pose))
    want = np.array([1.0, 0.5, 0.25, 0.25]) / 2.0
    np.testing.assert_allclose(sk["ubar"][0], want, rtol=1e-13)
    np.testing.assert_allclose(sk["ag"][0], want @ av.av[nb], rtol=1e-13)
    np.testing.assert_allclose(sk["rg"][0], want @ av.rv[nb], rtol=1e-13)
    np.testing.assert_allclose(sk["pg"][0], want @ av.pv[nb], rtol=1e-13)
    np.testing.assert_allclose(sk["wg"][0], want @ av.wv[nb], rtol=1e-12, atol=1e-15)


def test_skin_covariance_of_a_known_rotation(small_avatar):
    """Sigma = R(q) S^2 R(q)^T, q = (w, x, y, z) in the 3DGS convention:
    q = (cos t/2, 0, 0, sin t/2) turns by +t about +z.  At t = 45 degrees with
    scales s1 != s2 the xy term is (s1^2 - s2^2) / 2 (its sign fixes the
    direction of the turn); a quaternion of norm 3 gives the same (identity
    pose, so the blended transform is the identity)."""
    av = copy.deepcopy(small_avatar)
    av.pose = np.zeros((24, 3))
    s = np.array([0.02, 0.005, 0.01])
    q = np.array([math.cos(math.pi / 8), 0.0, 0.0, math.sin(math.pi / 8)])
    av.logscale[0] = av.logscale[1] = np.log(s)
    av.quat[0], av.quat[1] = q, 3.0 * q
    sk = O.skin(av, O.fk(av.parents, av.joints, av.pose))
    a, b, c = s ** 2
    want = [(a + b) / 2, (a - b) / 2, 0.0, (a + b) / 2, 0.0, c]
    for g in (0, 1):
        np.testing.assert_allclose(sk["cov"][g], want, rtol=1e-12, atol=1e-19)


def test_skin_displacement_moves_vertices_and_gaussians(small_avatar):
    """The displacement is interpolated by Eq. 1 like every attribute, and
    skinning moves x + dx: at the identity pose xp = x_v + dx_v and
    x_gd = x_g + sum_j ubar_j dx_j (ubar pinned above)."""
    av = copy.deepcopy(small_avatar)
    av.pose = np.zeros((24, 3))
    av.dxv = np.random.default_rng(8).normal(scale=0.01, size=av.xv.shape)
    sk = O.skin(av, O.fk(av.parents, av.joints, av.pose))
    np.testing.assert_allclose(sk["xp"], av.xv + av.dxv, atol=1e-14)
    want = av.xg + np.einsum("gk,gkc->gc", sk["ubar"], av.dxv[av.knn])
    np.testing.assert_allclose(sk["xd"], want, atol=1e-14)


def test_skin_normals_under_a_blended_pose(small_avatar):
    """Under a pose whose blended transforms are not rotations (the avatar's
    random +-30 degree pose), n_gd is still a unit vector along M n_g with M
    the blended linear part sum_k w_gk G_k and n_g = normalize(sum_j ubar_j
    n_j) (Eq. 1; w_g and ubar pinned above)."""
    av = small_avatar
    bone = O.fk(av.parents, av.joints, av.pose)
    sk = O.skin(av, bone)
    nbar = np.einsum("gk,gkc->gc", sk["ubar"], av.nv[av.knn])
    M = np.einsum("gk,kij->gij", sk["wg"], bone[:, :, :3])
    m = np.einsum("gij,gj->gi", M, nbar)
    assert np.max(np.abs(np.linalg.norm(m, axis=1) / np.linalg.norm(nbar, axis=1) - 1)) > 1e-3   # not rotations
    np.testing.assert_allclose(np.linalg.norm(sk["nd"], axis=1), 1.0, atol=1e-14)
    np.testing.assert_allclose(sk["nd"], m / np.linalg.norm(m, axis=1, keepdims=True), atol=1e-13)


def test_skin_identity_pose(small_avatar):
    av = copy.deepcopy(small_avatar)
    av.pose = np.zeros((24, 3))
    bone = O.fk(av.parents, av.joints, av.pose)
    sk = O.skin(av, bone)
    np.testing.assert_allclose(sk["xd"], av.xg, atol=1e-14)
    np.testing.assert_allclose(sk["xp"], av.xv, atol=1e-14)
    # covariance eigen-structure: eigenvalues exp(2 s), eigenvectors = rotation columns
    for g in range(0, av.G, 37):
        c = sk["cov"][g]
        S = np.array([[c[0], c[1], c[2]], [c[1], c[3], c[4]], [c[2], c[4], c[5]]])
        ev = np.sort(np.linalg.eigvalsh(S))
        np.testing.assert_allclose(ev, np.sort(np.exp(2 * av.logscale[g])), rtol=1e-10)
    # interpolated attributes stay inside the range of the neighbours
    for name, vert in (("ag", av.av), ("rg", av.rv), ("pg", av.pv)):
        nb = vert[av.knn]
        assert np.all(sk[name] >= nb.min(axis=1) - 1e-12)
        assert np.all(sk[name] <= nb.max(axis=1) + 1e-12)
    np.testing.assert_allclose(np.linalg.norm(sk["nd"], axis=1), 1, atol=1e-14)
    np.testing.assert_allclose(sk["wg"].sum(axis=1), 1, atol=1e-12)
    np.testing.assert_allclose(sk["ubar"].sum(axis=1), 1, atol=1e-14)


def test_skin_rigid_motion(small_avatar):
    av = copy.deepcopy(small_avatar)
    av.pose = np.zeros((24, 3))
    sk0 = O.skin(av, O.fk(av.parents, av.joints, av.pose))
    av.pose[0] = [0.3, 0.5, -0.2]
    Q = rot(av.pose[0], np.linalg.norm(av.pose[0]))
    J0 = av.joints[0]
    sk = O.skin(av, O.fk(av.parents, av.joints, av.pose))
    np.testing.assert_allclose(sk["xd"], (av.xg - J0) @ Q.T + J0, atol=1e-12)
    np.testing.assert_allclose(sk["nd"], sk0["nd"] @ Q.T, atol=1e-12)
    for g in range(0, av.G, 23):
        c0 = sk0["cov"][g]
        S0 = np.array([[c0[0], c0[1], c0[2]], [c0[1], c0[3], c0[4]], [c0[2], c0[4], c0[5]]])
        S1 = Q @ S0 @ Q.T
        np.testing.assert_allclose(sk["cov"][g], S1[[0, 0, 0, 1, 1, 2], [0, 1, 2, 1, 2, 2]],
                                   rtol=1e-10, atol=1e-16)


def test_skin_eq1_on_a_vertex_and_equidistant(small_avatar):
    av = copy.deepcopy(small_avatar)
    av.pose = np.zeros((24, 3))
    # Gaussian 0 sits on its first neighbour: Eq. 1 weight 1/d dominates
    av.xg[0] = av.xv[av.knn[0, 0]]
    # Gaussian 1: neighbours forced equidistant by placing it at their centroid
    # of a symmetric configuration (all K neighbours = the same vertex index)
    av.knn[1, :] = av.knn[1, 0]
    sk = O.skin(av, O.fk(av.parents, av.joints, av.pose))
    v0 = av.knn[0, 0]
    np.testing.assert_allclose(sk["ag"][0], av.av[v0], atol=1e-6)
    np.testing.assert_allclose(sk["rg"][0], av.rv[v0], atol=1e-6)
    v1 = av.knn[1, 0]
    np.testing.assert_allclose(sk["ag"][1], av.av[v1], atol=1e-14)
    np.testing.assert_allclose(sk["ubar"][1], 1.0 / av.K, atol=1e-15)


# ---------------------------------------------------------------- visibility
def _frames_for(dirs):
    return synth.direction_frames(np.asarray(dirs, float)).astype(np.float32).astype(np.float64)


def test_visibility_single_triangle_visible_from_both_sides():
    # nothing occludes a lone triangle: with the 2-pixel depth bias every vertex
    # is visible from every direction that is not within ~70 degrees of edge-on
    xp = np.array([[0.0, 0, 0], [0.3, 0, 0], [0, 0.3, 0]])
    faces = np.array([[0, 1, 2]], np.int32)
    dirs = synth.fibonacci_directions(64)
    R, half = 64, 1.0
    bits = O.visibility(xp, faces, _frames_for(dirs), [0.1, 0.1, 0], half, 2 * (2 * half / R), R)
    vb = np.unpackbits(bits.view(np.uint8), bitorder="little").reshape(3, 64)
    facing = np.abs(dirs[:, 2]) >= 0.35
    assert np.all(vb[:, facing] == 1)
    # and with no triangle at all every vertex is visible from everywhere
    bits = O.visibility(xp, np.zeros((0, 3), np.int32), _frames_for(dirs), [0.1, 0.1, 0], half,
                        0.0, R)
    assert np.all(bits == 0xFFFFFFFF)


def test_visibility_parallel_quads_occlusion():
    # near quad at z=+0.2 (spans [-0.5,0.5]^2), far quad at z=-0.2 (spans [0,1]x[-0.5,0.5])
    def quad(x0, x1, y0, y1, z, n):
        xs = np.linspace(x0, x1, n)
        ys = np.linspace(y0, y1, n)
        X, Y = np.meshgrid(xs, ys)
        v = np.stack([X.ravel(), Y.ravel(), np.full(X.size, z)], 1)
        f = []
        for j in range(n - 1):
            for i in range(n - 1):
                a = j * n + i
                f += [(a, a + 1, a + n), (a + 1, a + n + 1, a + n)]
        return v, np.array(f, np.int32)
    v1, f1 = quad(-0.5, 0.5, -0.5, 0.5, 0.2, 9)
    v2, f2 = quad(0.0, 1.0, -0.5, 0.5, -0.2, 9)
    xp = np.concatenate([v1, v2])
    faces = np.concatenate([f1, f2 + len(v1)])
    dirs = np.zeros((32, 3))
    dirs[:, 2] = 1.0                     # direction 0..31: light straight above (+z)
    dirs[16:, 2] = -1.0                  # 16..31: light straight below
    bits = O.visibility(xp, faces, _frames_for(dirs), [0.25, 0, 0], 1.2, 0.02, 128)
    b = bits[:, 0]
    up = (b & 1) != 0
    down = ((b >> 16) & 1) != 0
    n1 = len(v1)
    assert np.all(up[:n1])                                  # near quad lit from above
    far = v2
    inside = (far[:, 0] < 0.5 - 0.02) & (np.abs(far[:, 1]) < 0.5 - 0.02)
    outside = far[:, 0] > 0.5 + 0.02
    assert np.all(~up[n1:][inside])                         # shadowed by the near quad
    assert np.all(up[n1:][outside])
    assert np.all(down[n1:])                                # far quad lit from below
    near_inside = (v1[:, 0] > 0.02) & (np.abs(v1[:, 1]) < 0.5 - 0.02)
    assert np.all(~down[:n1][near_inside])


def test_visibility_convex_sphere_hemisphere():
    v, f, n = synth._tessellate_capsule((0, 0, 0), (0, 0, 0), 0.5, 2000)
    dirs = synth.fibonacci_directions(128)
    R = 256
    half = 0.6
    bias = 2.0 * (2 * half / R)
    bits = O.visibility(v, f, _frames_for(dirs), [0, 0, 0], half, bias, R)
    vb = np.unpackbits(bits.view(np.uint8), bitorder="little").reshape(len(v), -1)[:, :128]
    cosines = n @ dirs.T
    tau = 0.35
    assert np.all(vb[cosines >= tau] == 1)
    assert np.all(vb[cosines <= -tau] == 0)


def test_visibility_one_sided_equals_two_sided_on_a_closed_mesh():
    # the capsule body is a union of watertight, outward-wound meshes: the
    # nearest surface along any ray toward a light faces that light, so
    # rasterising only light-facing triangles gives the same depth maps
    sc = synth.config_scene("c1_small", n_dirs=64, depth_res=128)
    av = sc.avatar
    sk = O.skin(av, O.fk(av.parents, av.joints, av.pose))
    xp = np.asarray(sk["xp"], np.float32).astype(np.float64)
    fr = np.asarray(sc.frames.reshape(-1, 9), np.float32).astype(np.float64)
    args = (xp, av.faces, fr, sc.window_center, sc.window_half, sc.vis_bias, sc.depth_res)
    b2, d2 = O.visibility(*args, want_depth=True)
    b1, d1 = O.visibility(*args, want_depth=True, cull_back=True)
    assert np.array_equal(d1, d2)
    assert np.array_equal(b1, b2)
    # but not on an open surface seen from behind: a lone triangle casts no
    # shadow from its back side when culled
    tri = np.array([[0.0, 0, 0], [0.3, 0, 0], [0, 0.3, 0]])
    dirs = np.array([[0, 0, -1.0]] * 32)
    _, dd = O.visibility(tri, np.array([[0, 1, 2]], np.int32), _frames_for(dirs), [0.1, 0.1, 0], 1.0, 0.0,
                         64, want_depth=True, cull_back=True)
    assert np.all(dd == np.iinfo(np.int32).max)


def test_visibility_depth_map_of_a_plane():
    # one big triangle facing +z; depth at each covered pixel centre equals the
    # plane's depth (zd = -z * 2^16) up to the integer floor and quantisation.
    xp = np.array([[-0.5, -0.5, 0.1], [0.5, -0.5, 0.3], [-0.5, 0.5, -0.1]])
    faces = np.array([[0, 1, 2]], np.int32)
    dirs = np.zeros((32, 3))
    dirs[:, 2] = 1
    fr = _frames_for(dirs)
    R = 64
    half = 0.75
    bits, depth = O.visibility(xp, faces, fr, [0, 0, 0], half, 0.0, R, want_depth=True)
    e1, e2, w = fr[0].reshape(3, 3)
    d0 = depth[0]
    covered = d0 != np.iinfo(np.int32).max
    assert covered.sum() > 0.15 * R * R      # the triangle covers 2/9 of the window
    # plane z(x,y) through the three vertices
    A = np.c_[xp[:, :2], np.ones(3)]
    coef = np.linalg.solve(A, xp[:, 2])
    jj, ii = np.nonzero(covered)
    # pixel centre -> s, t world coordinates in the frame basis
    s = (ii + 0.5) / R * 2 * half - half
    t = (jj + 0.5) / R * 2 * half - half
    P = np.outer(s, e1) + np.outer(t, e2)
    z = coef[0] * P[:, 0] + coef[1] * P[:, 1] + coef[2]
    expect = -z * 65536.0
    assert np.max(np.abs(d0[jj, ii] - expect)) < 40.0   # ~0.6 mm: fixed-point steps


def test_visibility_covers_exactly_the_pixel_centres_inside():
    """A triangle covers a depth-map pixel iff the pixel's centre lies inside
    it (all three edge functions >= 0): compared with an FP64 barycentric
    test of every centre, leaving out centres within 0.1 pixel of an edge
    (the vertices are placed in 1/16-pixel steps, which decide those)."""
    xp = np.array([[-0.41, -0.37, 0.0], [0.45, -0.12, 0.1], [-0.08, 0.43, -0.1]])
    faces = np.array([[0, 1, 2]], np.int32)
    dirs = np.zeros((32, 3))
    dirs[:, 2] = 1
    fr = _frames_for(dirs)
    R, half = 64, 0.75
    _, depth = O.visibility(xp, faces, fr, [0, 0, 0], half, 0.0, R, want_depth=True)
    covered = depth[0] != np.iinfo(np.int32).max
    e1, e2, _ = fr[0].reshape(3, 3)
    st = np.c_[xp @ e1, xp @ e2] / (2 * half / R)            # vertices in pixel units
    st += R / 2
    jj, ii = np.mgrid[0:R, 0:R]
    P = np.stack([ii + 0.5, jj + 0.5], -1)

    def edge(a, b):
        d = st[b] - st[a]
        return (d[0] * (P[..., 1] - st[a][1]) - d[1] * (P[..., 0] - st[a][0])) / np.hypot(*d)
    E = np.stack([edge(1, 2), edge(2, 0), edge(0, 1)])
    if np.sum(E > 0) < np.sum(E < 0):
        E = -E
    inside = np.all(E >= 0, axis=0)
    sure = np.all(np.abs(E) > 0.1, axis=0)
    assert inside.sum() > 300
    np.testing.assert_array_equal(covered[sure], inside[sure])


def test_visibility_rejects_unsupported_arguments():
    xp = np.zeros((3, 3))
    faces = np.array([[0, 1, 2]], np.int32)
    with pytest.raises(ValueError):
        O.visibility(xp, faces, _frames_for(np.eye(3)[[2] * 30]), [0, 0, 0], 1.0, 0.0, 64)
    with pytest.raises(ValueError):
        O.visibility(xp, faces, _frames_for(np.eye(3)[[2] * 32]), [0, 0, 0], 1.0, 0.0, 2048)
    with pytest.raises(ValueError):
        O.visibility(np.full((3, 3), 9.0), faces, _frames_for(np.eye(3)[[2] * 32]), [0, 0, 0],
                     1.0, 0.0, 64)


# ---------------------------------------------------------------- shading
def _one_gaussian(n, x=(0, 0, 0), a=(0.5, 0.5, 0.5), rough=0.5, spec=0.0):
    return (np.array([x], float), np.array([n], float), np.array([a], float),
            np.array([rough]), np.array([spec]), np.ones((1, 1)), np.zeros((1, 1), np.int32))


def test_light_solid_angles_and_quadrature():
    rng = np.random.default_rng(0)
    for rows, cols in ((8, 16), (16, 32), (32, 64)):
        lt = synth.latlong_light(rng, rows, cols)
        assert abs(lt.A.sum() - 4 * math.pi) < 1e-12
    lt = synth.latlong_light(rng, 32, 64)
    for n in ([0, 1, 0], [1, 0, 0], [0.3, -0.5, 0.8]):
        n = np.array(n) / np.linalg.norm(n)
        Q = np.sum(lt.A * np.maximum(0, lt.w @ n))
        assert abs(Q - math.pi) < 0.01


def test_shade_lambertian_constant_light_all_visible():
    """Constant L, full visibility, p = 0: colour = (a L Q(n)/pi)^(1/2.2)."""
    rng = np.random.default_rng(1)
    lt = synth.latlong_light(rng, 16, 32)
    Lc = np.full_like(lt.L, 1.7)
    dmap = np.arange(len(lt.A), dtype=np.int32) % 32
    bits = np.full((1, 1), 0xFFFFFFFF, np.uint32)
    for n in ([0, 0, 1], [0.6, 0.0, 0.8], [0.1, 0.9, 0.3]):
        n = np.array(n) / np.linalg.norm(n)
        xd, nd, a, r, p, ub, knn = _one_gaussian(n, a=(0.2, 0.5, 0.9))
        cam = 10.0 * n
        col, rad, cull = O.shade(xd, nd, a, r, p, ub, knn, bits, Lc, lt.A, lt.w, dmap, cam, 32)
        Q = np.sum(lt.A * np.maximum(0, lt.w @ n))
        np.testing.assert_allclose(rad[0], a[0] * 1.7 * Q / math.pi, rtol=1e-13)
        np.testing.assert_allclose(col[0], (a[0] * 1.7 * Q / math.pi) ** (1 / 2.2), rtol=1e-13)
        # albedo x L within the quadrature error of the 16x32 light
        np.testing.assert_allclose(rad[0], a[0] * 1.7, rtol=0.02)
        assert cull[0] == 0


def test_shade_visibility_is_linear_in_the_bits():
    rng = np.random.default_rng(2)
    lt = synth.latlong_light(rng, 8, 16)
    dmap = np.arange(128, dtype=np.int32)
    n = np.array([0.2, 0.7, 0.3])
    n /= np.linalg.norm(n)
    xd, nd, a, r, p, ub, knn = _one_gaussian(n, spec=0.7, rough=0.4)
    cam = 5.0 * np.array([0.3, 0.8, 0.4])
    mask = rng.integers(0, 2 ** 32, size=(1, 4), dtype=np.uint64).astype(np.uint32)
    full = np.full((1, 4), 0xFFFFFFFF, np.uint32)
    _, r_all, _ = O.shade(xd, nd, a, r, p, ub, knn, full, lt.L, lt.A, lt.w, dmap, cam, 128)
    _, r_m, _ = O.shade(xd, nd, a, r, p, ub, knn, mask, lt.L, lt.A, lt.w, dmap, cam, 128)
    _, r_c, _ = O.shade(xd, nd, a, r, p, ub, knn, ~mask, lt.L, lt.A, lt.w, dmap, cam, 128)
    np.testing.assert_allclose(r_m + r_c, r_all, rtol=1e-13)
    # two neighbours with weights 0.25/0.75 and complementary bits: vis = 0.25 / 0.75
    ub2 = np.array([[0.25, 0.75]])
    knn2 = np.array([[0, 1]], np.int32)
    bits2 = np.concatenate([mask, ~mask])
    _, r_mix, _ = O.shade(xd, nd, a, r, p, ub2, knn2, bits2, lt.L, lt.A, lt.w, dmap, cam, 128)
    np.testing.assert_allclose(r_mix, 0.25 * r_m + 0.75 * r_c, rtol=1e-13)


def test_shade_light_reads_the_bit_of_its_viewpoint():
    """Light k takes bit d(k) = dmap[k] of each neighbour's words (word d/32,
    bit d%32).  One light whose viewpoint is direction 77 of 128 is lit with
    bit 77 alone set and dark with every bit but 77; and shading under a
    permuted dmap equals shading under the identity map of words whose bit k
    is bit dmap[k] of the original."""
    n = np.array([0.3, 0.2, 0.9])
    n /= np.linalg.norm(n)
    xd, nd, a, r, p, ub, knn = _one_gaussian(n, spec=0.5)
    cam = 4.0 * n
    L, A, w = np.array([[1.0, 0.5, 0.25]]), np.array([0.1]), n[None]
    only = np.zeros((1, 4), np.uint32)
    only[0, 77 // 32] = np.uint32(1 << (77 % 32))
    _, lit, _ = O.shade(xd, nd, a, r, p, ub, knn, only, L, A, w, np.array([77], np.int32), cam, 128)
    _, dark, _ = O.shade(xd, nd, a, r, p, ub, knn, ~only, L, A, w, np.array([77], np.int32), cam, 128)
    _, full, _ = O.shade(xd, nd, a, r, p, ub, knn, np.full((1, 4), 0xFFFFFFFF, np.uint32), L, A, w,
                         np.array([77], np.int32), cam, 128)
    assert np.all(lit[0] > 0) and np.all(dark[0] == 0)
    np.testing.assert_array_equal(lit, full)
    rng = np.random.default_rng(9)
    lt = synth.latlong_light(rng, 8, 16)
    perm = rng.permutation(128).astype(np.int32)
    words = rng.integers(0, 2 ** 32, size=(1, 4), dtype=np.uint64).astype(np.uint32)
    bitv = np.unpackbits(words.view(np.uint8), bitorder="little")
    moved = np.packbits(bitv[perm], bitorder="little").view(np.uint32)[None]
    _, r1, _ = O.shade(xd, nd, a, r, p, ub, knn, words, lt.L, lt.A, lt.w, perm, cam, 128)
    _, r2, _ = O.shade(xd, nd, a, r, p, ub, knn, moved, lt.L, lt.A, lt.w, np.arange(128, dtype=np.int32), cam, 128)
    np.testing.assert_allclose(r1, r2, rtol=1e-13)


def test_shade_normal_incidence_closed_form():
    """Light, view and normal aligned: f_s = F(1) / (4 pi alpha^2), App. A."""
    gc = golden_constants()
    n = np.array([0.0, 0.0, 1.0])
    for gamma in (0.3, 0.55, 0.9):
        xd, nd, a, r, p, ub, knn = _one_gaussian(n, a=(0, 0, 0), rough=gamma, spec=1.0)
        L = np.array([[1.0, 2.0, 3.0]])
        A = np.array([0.01])
        w = np.array([n])
        cam = 1e7 * n
        _, rad, _ = O.shade(xd, nd, a, r, p, ub, knn, np.full((1, 1), 1, np.uint32), L, A, w,
                            np.zeros(1, np.int32), cam, 32)
        alpha = gamma ** gc["alpha_power"]
        F = gc["F0"] + (1 - gc["F0"]) * 2.0 ** ((gc["fresnel_a"] + gc["fresnel_b"]))
        fs = F / (4 * math.pi * alpha * alpha)
        np.testing.assert_allclose(rad[0], L[0] * A[0] * fs, rtol=1e-9)


def test_shade_brdf_reciprocity_and_furnace_bound():
    n = np.array([0.0, 1.0, 0.0])
    rng = np.random.default_rng(3)
    for _ in range(6):
        w1 = rng.normal(size=3); w1[1] = abs(w1[1]) + 0.1; w1 /= np.linalg.norm(w1)
        w2 = rng.normal(size=3); w2[1] = abs(w2[1]) + 0.1; w2 /= np.linalg.norm(w2)
        gamma = rng.uniform(0.3, 0.9)
        xd, nd, a, r, p, ub, knn = _one_gaussian(n, a=(0, 0, 0), rough=gamma, spec=1.0)
        one = np.ones((1, 3))
        bits = np.full((1, 1), 1, np.uint32)
        z = np.zeros(1, np.int32)
        _, r12, _ = O.shade(xd, nd, a, r, p, ub, knn, bits, one, np.ones(1), w1[None], z, 1e7 * w2, 32)
        _, r21, _ = O.shade(xd, nd, a, r, p, ub, knn, bits, one, np.ones(1), w2[None], z, 1e7 * w1, 32)
        np.testing.assert_allclose(r12 / (n @ w1), r21 / (n @ w2), rtol=1e-6)
    # white furnace: specular directional albedo never exceeds 1
    lt = synth.latlong_light(rng, 64, 128)
    full = np.full((1, 256), 0xFFFFFFFF, np.uint32)
    dmap = np.arange(len(lt.A), dtype=np.int32) % 8192
    for gamma in (0.3, 0.6, 0.9):
        for th in (0.0, 0.7, 1.3):
            wo = np.array([math.sin(th), math.cos(th), 0.0])
            xd, nd, a, r, p, ub, knn = _one_gaussian(n, a=(0, 0, 0), rough=gamma, spec=1.0)
            _, rad, _ = O.shade(xd, nd, a, r, p, ub, knn, full, np.ones_like(lt.L), lt.A, lt.w,
                                dmap, 1e7 * wo, 8192)
            assert 0.0 < rad[0, 0] <= 1.0


# ---------------------------------------------------------------- App. A terms against mathematics
def _check_ggx_normalised(brdf):
    """A microfacet distribution has unit projected area: the integral of
    D(h) (n.h) over the hemisphere of h is 1.  With mu = n.h and t = mu^2 the
    integral 2 pi int_0^1 D(mu) mu dmu becomes pi int_0^1 D(sqrt t) dt, taken
    by adaptive FP64 quadrature (breakpoints where the lobe of width ~alpha^2
    sits)."""
    from scipy import integrate
    for gamma in (0.3, 0.6, 0.9):
        a2 = gamma ** 4
        val, _ = integrate.quad(lambda t: brdf(gamma, math.sqrt(t), 1.0, 1.0, 1.0)[0], 0.0, 1.0, limit=400,
                                epsabs=1e-13, epsrel=1e-11, points=[1.0 - a2, 1.0 - 10.0 * a2])
        assert abs(math.pi * val - 1.0) < 1e-8, f"gamma {gamma}: projected area {math.pi * val}"


def _check_smith_g1(brdf):
    """G1 by hand from App. A's k = (gamma + 1)^2 / 8 and G1(c) = c / (c (1 - k) + k):
    gamma = 1/2: k = 9/32, G1(1/2) = (1/2) / (23/64 + 18/64) = 32/41;
    gamma = 0.9: k = 361/800, G1(1/2) = (1/2) / (439/1600 + 722/1600) = 800/1161;
    G1(1) = 1 for every k, so G(1/2, 1) = G1(1/2) and G(1/2, 1/2) = G1(1/2)^2."""
    for gamma, g1 in ((0.5, 32.0 / 41.0), (0.9, 800.0 / 1161.0)):
        assert abs(brdf(gamma, 1.0, 1.0, 0.5, 1.0)[2] - g1) < 1e-14, gamma
        assert abs(brdf(gamma, 1.0, 1.0, 1.0, 0.5)[2] - g1) < 1e-14, gamma
        assert abs(brdf(gamma, 1.0, 1.0, 0.5, 0.5)[2] - g1 * g1) < 1e-14, gamma
        assert abs(brdf(gamma, 1.0, 1.0, 1.0, 1.0)[2] - 1.0) < 1e-15, gamma


def _check_fresnel_schlick(brdf):
    """App. A's Fresnel term is the spherical-Gaussian fit of Schlick's
    F0 + (1 - F0)(1 - x)^5 (x = w_o.h, F0 = 0.04): within 1e-2 of it over
    [0, 1] (the fit's worst case is 3.6e-3), exactly 1 at x = 0."""
    x = np.linspace(0.0, 1.0, 1001)
    F = np.array([brdf(0.5, 1.0, xi, 1.0, 1.0)[1] for xi in x])
    assert np.abs(F - (0.04 + 0.96 * (1.0 - x) ** 5)).max() < 1e-2
    assert F[0] == 1.0


def _check_cancelled_form(brdf):
    """The shading sums use f_s = D F / (4 (c_i(1-k)+k)(c_o(1-k)+k)); it must
    equal the printed D F G / (4 c_i c_o) with the pinned D, F, G wherever both
    cosines are positive."""
    rng = np.random.default_rng(4)
    for _ in range(50):
        gamma, nh, voh, ci, co = rng.uniform(0.3, 0.9), *rng.uniform(0.05, 1.0, size=4)
        D, F, G, fs = brdf(gamma, nh, voh, ci, co)
        assert abs(fs - D * F * G / (4.0 * ci * co)) <= 1e-12 * abs(fs)


BRDF_CHECKS = (_check_ggx_normalised, _check_smith_g1, _check_fresnel_schlick, _check_cancelled_form)


@pytest.mark.parametrize("check", BRDF_CHECKS, ids=lambda f: f.__name__[7:])
def test_brdf_terms_against_mathematics(check):
    check(lambda *a: O.brdf_terms(*a))


def test_shade_sums_the_pinned_brdf_terms():
    """One Gaussian, one light, albedo 0, tint 1: the radiance is
    L A c_i f_s with f_s the pinned App. A term at this geometry's cosines."""
    rng = np.random.default_rng(6)
    for _ in range(8):
        n = rng.normal(size=3); n /= np.linalg.norm(n)
        wi = rng.normal(size=3); wi += (0.3 - wi @ n) * n if wi @ n < 0.3 else 0; wi /= np.linalg.norm(wi)
        wo = rng.normal(size=3); wo += (0.3 - wo @ n) * n if wo @ n < 0.3 else 0; wo /= np.linalg.norm(wo)
        gamma = rng.uniform(0.3, 0.9)
        xd, nd, a, r, p, ub, knn = _one_gaussian(n, a=(0, 0, 0), rough=gamma, spec=1.0)
        L = np.array([[0.7, 1.1, 2.0]])
        A = np.array([0.02])
        _, rad, _ = O.shade(xd, nd, a, r, p, ub, knn, np.full((1, 1), 1, np.uint32), L, A, wi[None],
                            np.zeros(1, np.int32), 1e7 * wo, 32)
        h = (wi + wo) / np.linalg.norm(wi + wo)
        fs = O.brdf_terms(gamma, n @ h, wo @ h, n @ wi, n @ wo)[3]
        np.testing.assert_allclose(rad[0], L[0] * A[0] * (n @ wi) * fs, rtol=1e-6)


@pytest.mark.parametrize("old,new,expect", [
    ("kk = (gamma + 1.0) * (gamma + 1.0) / 8.0;", "kk = (gamma + 1.0) * (gamma + 1.0) / 4.0;", "smith_g1"),
    ("double den = nh * nh * (a2 - 1.0) + 1.0;", "double den = nh * (a2 - 1.0) + 1.0;", "ggx_normalised"),
    ("(-5.55473 * voh - 6.98316) * voh", "(-5.55473 * voh + 6.98316) * voh", "fresnel_schlick"),
    ("out[3] = Dn * Fr / (4.0 * gi * go);", "out[3] = Dn * Fr / (4.0 * gi);", "cancelled_form"),
], ids=["k_over_4", "D_linear_in_nh", "F_sign", "fs_drops_G1o"])
def test_brdf_pins_catch_planted_mistakes(tmp_path, old, new, expect):
    """Plants a plausible mistake in a copy of the oracle source (never in the
    oracle itself), builds it and checks that some App. A pin fails on it."""
    import ctypes
    import subprocess
    src = open(O._SRC).read()
    assert src.count(old) == 1
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-o", str(so),
                           str(path), "-lm"])
    mut = ctypes.CDLL(str(so))
    failed = []
    for check in BRDF_CHECKS:
        try:
            check(lambda *a: O.brdf_terms(*a, library=mut))
        except AssertionError:
            failed.append(check.__name__[7:])
    assert expect in failed, f"the {expect} pin passes the planted mistake {new!r} (failed: {failed})"


def test_shade_backface_cull():
    n = np.array([0.0, 0.0, 1.0])
    xd, nd, a, r, p, ub, knn = _one_gaussian(n)
    lt = synth.latlong_light(np.random.default_rng(0), 8, 16)
    dmap = np.zeros(128, np.int32)
    bits = np.full((1, 1), 1, np.uint32)
    col, rad, cull = O.shade(xd, nd, a, r, p, ub, knn, bits, lt.L, lt.A, lt.w, dmap,
                             np.array([0, 0, -3.0]), 32)
    assert cull[0] == 1 and np.all(col == 0)
    col, rad, cull = O.shade(xd, nd, a, r, p, ub, knn, bits, lt.L, lt.A, lt.w, dmap,
                             np.array([0, 0, 3.0]), 32)
    assert cull[0] == 0 and np.all(col > 0)


# ---------------------------------------------------------------- projection
def _cam(width=64, height=64, f=100.0, R=None, t=(0, 0, 0)):
    R = np.eye(3) if R is None else R
    t = np.asarray(t, float)
    return synth.Camera(fx=f, fy=f * 1.1, cx=width / 2, cy=height / 2, width=width, height=height,
                        R=R, t=t, center=-R.T @ t)


def test_project_isotropic_on_axis_closed_form():
    cam = _cam()
    sigma, z = 0.02, 2.0
    xd = np.array([[0.0, 0.0, z]])
    cov = np.array([[sigma ** 2, 0, 0, sigma ** 2, 0, sigma ** 2]])
    pr = O.project(xd, cov, np.array([0.8]), None, cam)
    sx = (cam.fx * sigma / z) ** 2 + 0.3
    sy = (cam.fy * sigma / z) ** 2 + 0.3
    np.testing.assert_allclose(pr["conic"][0], [1 / sx, 0, 1 / sy], rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose(pr["mean2d"][0], [cam.cx, cam.cy], atol=1e-13)
    assert pr["valid"][0] == 1 and pr["depth"][0] == z


def test_project_offaxis_matches_numeric_jacobian():
    rng = np.random.default_rng(4)
    R = rot([0.3, 1, 0.2], 0.4)
    cam = _cam(R=R, t=(0.1, -0.2, 3.0))
    for _ in range(5):
        x = rng.normal(scale=0.3, size=3)
        A = rng.normal(scale=0.03, size=(3, 3))
        S = A @ A.T
        cov = S[[0, 0, 0, 1, 1, 2], [0, 1, 2, 1, 2, 2]][None]
        pr = O.project(x[None], cov, np.array([0.9]), None, cam)

        def pix(y):
            p = R @ y + cam.t
            return np.array([cam.fx * p[0] / p[2] + cam.cx, cam.fy * p[1] / p[2] + cam.cy])
        h = 1e-6
        Jn = np.stack([(pix(x + h * e) - pix(x - h * e)) / (2 * h) for e in np.eye(3)], axis=1)
        S2 = Jn @ S @ Jn.T + 0.3 * np.eye(2)
        inv = np.linalg.inv(S2)
        np.testing.assert_allclose(pr["conic"][0], [inv[0, 0], inv[0, 1], inv[1, 1]], rtol=1e-6)
        np.testing.assert_allclose(pr["mean2d"][0], pix(x), rtol=1e-13)


def test_project_validity_rules():
    cam = _cam()
    xd = np.array([[0, 0, 0.1], [0, 0, 1.0], [0, 0, 1.0], [0, 0, 1.0]])
    cov = np.tile([[1e-4, 0, 0, 1e-4, 0, 1e-4]], (4, 1))
    op = np.array([0.5, 0.5, 0.5, 1.0 / 300])
    cull = np.array([0, 1, 0, 0], np.uint8)
    pr = O.project(xd, cov, op, cull, cam)
    assert list(pr["valid"]) == [0, 0, 1, 0]


def test_project_rect_contains_the_alpha_support():
    rng = np.random.default_rng(6)
    cam = _cam(width=96, height=80, f=120.0)
    G = 40
    xd = np.c_[rng.uniform(-0.3, 0.3, G), rng.uniform(-0.3, 0.3, G), rng.uniform(1.0, 2.0, G)]
    covs = []
    for _ in range(G):
        A = rng.normal(scale=0.03, size=(3, 3))
        S = A @ A.T
        covs.append(S[[0, 0, 0, 1, 1, 2], [0, 1, 2, 1, 2, 2]])
    op = rng.uniform(0.3, 0.95, G)
    pr = O.project(xd, np.array(covs), op, None, cam)
    ys, xs = np.mgrid[0:cam.height, 0:cam.width]
    for g in range(G):
        dx = xs + 0.5 - pr["mean2d"][g, 0]
        dy = ys + 0.5 - pr["mean2d"][g, 1]
        c = pr["conic"][g]
        a = op[g] * np.exp(-0.5 * (c[0] * dx * dx + 2 * c[1] * dx * dy + c[2] * dy * dy))
        jj, ii = np.nonzero(a >= 1 / 255)
        r = pr["rect"][g]
        assert np.all((ii >= r[0]) & (ii <= r[2]) & (jj >= r[1]) & (jj <= r[3]))


# ---------------------------------------------------------------- compositing
def test_composite_one_and_two_gaussians_closed_form():
    W = H = 16
    m = np.array([[8.0, 8.0], [8.5, 7.5]])
    conic = np.array([[0.05, 0.01, 0.04], [0.03, -0.005, 0.06]])
    op = np.array([0.7, 0.6])
    col = np.array([[1.0, 0.2, 0.1], [0.1, 0.3, 0.9]])
    px = np.array([7 * W + 9])
    x, y = 9.5, 7.5

    def alpha(g):
        dx, dy = x - m[g, 0], y - m[g, 1]
        c = conic[g]
        return min(0.99, op[g] * math.exp(-0.5 * (c[0] * dx * dx + 2 * c[1] * dx * dy + c[2] * dy * dy)))
    a0, a1 = alpha(0), alpha(1)
    rgb, T, cnt, _ = O.composite(m[:1], conic[:1], op[:1], col[:1], np.array([1.0]), [1], W, H, px)
    np.testing.assert_allclose(rgb[0], col[0] * a0, rtol=1e-14)
    np.testing.assert_allclose(T[0], 1 - a0, rtol=1e-14)
    for d in ([1.0, 2.0], [2.0, 1.0]):
        rgb, T, cnt, _ = O.composite(m, conic, op, col, np.array(d), [1, 1], W, H, px)
        f, b = (0, 1) if d[0] < d[1] else (1, 0)
        af, ab = (a0, a1) if f == 0 else (a1, a0)
        np.testing.assert_allclose(rgb[0], col[f] * af + col[b] * ab * (1 - af), rtol=1e-14)
        np.testing.assert_allclose(T[0], (1 - af) * (1 - ab), rtol=1e-14)
        assert cnt[0] == 2


def test_composite_alpha_is_clamped_at_0_99():
    """An opaque Gaussian (o = 1) centred on a pixel centre: alpha =
    min(0.99, 1) = 0.99, so that pixel's colour is 0.99 c and T = 0.01."""
    col = np.array([[0.4, 0.8, 0.2]])
    rgb, T, cnt, _ = O.composite(np.array([[8.5, 8.5]]), np.array([[0.2, 0.0, 0.2]]), np.array([1.0]), col,
                                 np.array([1.0]), [1], 16, 16, np.array([8 * 16 + 8]))
    np.testing.assert_allclose(rgb[0], 0.99 * col[0], rtol=1e-15)
    np.testing.assert_allclose(T[0], 0.01, rtol=1e-13)
    assert cnt[0] == 1


def test_composite_weights_sum_to_at_most_one_and_stop_rule():
    sc = synth.config_scene("c3_fd")
    fr = OP.frame(sc)
    pr = fr["proj"]
    ones = np.ones_like(fr["color"])
    rgb, T, cnt, amb = O.composite(pr["mean2d"], pr["conic"], sc.avatar.opacity, ones,
                                   pr["depth"], pr["valid"], 64, 64)
    np.testing.assert_allclose(rgb[:, 0], 1 - T, atol=1e-12)
    assert np.all(T >= 1e-4 - 1e-15) and np.all(T <= 1.0)
    # a stack of opaque Gaussians stops once T would drop below 1e-4
    n = 12
    m = np.tile([[8.0, 8.0]], (n, 1))
    conic = np.tile([[1e-4, 0, 1e-4]], (n, 1))
    op = np.full(n, 0.9)
    rgb, T, cnt, _ = O.composite(m, conic, op, np.ones((n, 3)), np.arange(n, dtype=float),
                                 np.ones(n), 16, 16, np.array([8 * 16 + 8]))
    a = 0.9 * math.exp(-0.5 * 1e-4 * 0.5)
    k = 0
    t = 1.0
    while t * (1 - a) >= 1e-4:
        t *= 1 - a
        k += 1
    assert cnt[0] == k
    np.testing.assert_allclose(T[0], t, rtol=1e-13)


# ---------------------------------------------------------------- binning
def test_bin_matches_pairwise_enumeration():
    rng = np.random.default_rng(7)
    G, W, H, TS = 300, 100, 70, 16
    x0 = rng.integers(-5, W, G); y0 = rng.integers(-5, H, G)
    x1 = x0 + rng.integers(-3, 40, G); y1 = y0 + rng.integers(-3, 30, G)
    rect = np.c_[np.clip(x0, 0, W - 1), np.clip(y0, 0, H - 1), np.clip(x1, 0, W - 1), np.clip(y1, 0, H - 1)]
    rect[x1 < 0] = [0, 0, -1, -1]
    key = rng.integers(0, 50, G).astype(np.uint32)     # many equal keys: tests the index tie-break
    start, lst = O.bin_tiles(rect, key, W, H, TS)
    tx = (W + TS - 1) // TS
    pairs = []
    for g in range(G):
        r = rect[g]
        if r[0] > r[2] or r[1] > r[3]:
            continue
        for ty in range(r[1] // TS, r[3] // TS + 1):
            for txx in range(r[0] // TS, r[2] // TS + 1):
                pairs.append((ty * tx + txx, int(key[g]), g))
    pairs.sort()
    assert len(pairs) == len(lst)
    assert [p[2] for p in pairs] == list(lst)
    counts = np.bincount([p[0] for p in pairs], minlength=len(start) - 1)
    np.testing.assert_array_equal(np.diff(start), counts)


# ---------------------------------------------------------------- adjoint
def _fd_setup():
    sc = synth.config_scene("c3_fd")
    fr = OP.frame(sc)
    av = sc.avatar
    fixed = dict(knn=av.knn, xv=AJ.t64(av.xv), dxv=AJ.t64(av.dxv), nv=AJ.t64(av.nv),
                 bone=AJ.t64(fr["bone"]), bits=fr["bits"], dmap=sc.dmap, A=AJ.t64(sc.light.A),
                 w=AJ.t64(sc.light.w), cam_center=AJ.t64(sc.camera.center), culled=fr["cull"],
                 valid=fr["proj"]["valid"], cam=sc.camera)
    params = dict(xg=av.xg, logscale=av.logscale, quat=av.quat, opacity=av.opacity, av=av.av,
                  rv=av.rv, pv=av.pv, L=sc.light.L, wv=av.wv)
    return sc, fr, fixed, params


def test_adjoint_forward_agrees_with_c_oracle():
    sc, fr, fixed, params = _fd_setup()
    tp = {k: AJ.t64(v) for k, v in params.items()}
    img = AJ.render(tp, fixed).numpy().reshape(-1, 3)
    ok = fr["amb"] == 0
    assert ok.mean() > 0.98
    np.testing.assert_allclose(img[ok], fr["rgb"][ok], atol=1e-11)


def _c_loss(sc, fr, params, target):
    s2 = copy.deepcopy(sc)
    av = s2.avatar
    av.xg, av.logscale, av.quat, av.opacity = params["xg"], params["logscale"], params["quat"], params["opacity"]
    av.av, av.rv, av.pv, av.wv = params["av"], params["rv"], params["pv"], params["wv"]
    s2.light.L = params["L"]
    out = OP.frame(s2, bits=fr["bits"])
    return np.abs(out["rgb"] - target).mean()


def test_adjoint_matches_central_finite_differences():
    sc, fr, fixed, params = _fd_setup()
    rng = np.random.default_rng(11)
    # target: the same frame with perturbed albedo, roughness and light
    tgt_params = dict(params)
    tgt_params["av"] = np.clip(params["av"] * rng.uniform(0.8, 1.2, params["av"].shape), 0, 1)
    tgt_params["rv"] = np.clip(params["rv"] + rng.normal(0, 0.05, params["rv"].shape), 0.2, 1)
    tgt_params["L"] = params["L"] * rng.uniform(0.8, 1.2, params["L"].shape)
    s_t = copy.deepcopy(sc)
    s_t.avatar.av, s_t.avatar.rv, s_t.light.L = tgt_params["av"], tgt_params["rv"], tgt_params["L"]
    target = OP.frame(s_t, bits=fr["bits"])["rgb"]
    tp = {k: AJ.t64(v).requires_grad_(True) for k, v in params.items()}
    img = AJ.render(tp, fixed)
    loss = AJ.l1_loss(img, AJ.t64(target).reshape(img.shape))
    loss.backward()
    valid = np.nonzero(fr["proj"]["valid"])[0]
    used_v = np.unique(sc.avatar.knn[valid])
    picks = {
        "xg": [(g, c) for g in rng.choice(valid, 4) for c in (rng.integers(3),)],
        "logscale": [(g, rng.integers(3)) for g in rng.choice(valid, 4)],
        "quat": [(g, rng.integers(4)) for g in rng.choice(valid, 4)],
        "opacity": [(g,) for g in rng.choice(valid, 4)],
        "av": [(v, rng.integers(3)) for v in rng.choice(used_v, 4)],
        "rv": [(v,) for v in rng.choice(used_v, 4)],
        "pv": [(v,) for v in rng.choice(used_v, 4)],
        "L": [(k, rng.integers(3)) for k in rng.integers(0, len(sc.light.A), 4)],
        "wv": [(v, rng.integers(24)) for v in rng.choice(used_v, 4)],
    }
    kinks = 0
    for name, idxs in picks.items():
        g_all = tp[name].grad.numpy()
        for idx in idxs:
            idx = tuple(int(i) for i in idx)
            base = params[name]
            h = 1e-6 * max(1.0, abs(float(base[idx])))
            def fd(step):
                p_plus = dict(params); p_minus = dict(params)
                a = base.copy(); a[idx] += step; p_plus[name] = a
                b = base.copy(); b[idx] -= step; p_minus[name] = b
                return (_c_loss(sc, fr, p_plus, target) - _c_loss(sc, fr, p_minus, target)) / (2 * step)
            d1 = fd(h)
            ga = float(g_all[idx])
            if abs(d1 - ga) <= 1e-5 * max(abs(d1), abs(ga)) + 1e-10:
                continue
            d2 = fd(h / 4)
            if abs(d1 - d2) > 1e-4 * max(abs(d1), 1e-8):   # threshold crossing: not a smooth point
                kinks += 1
                continue
            raise AssertionError(f"{name}{idx}: autograd {ga} vs FD {d1}")
    assert kinks <= 2


def test_bf16_rounding_helper_matches_torch():
    """The tests' BF16 rounding of oracle inputs equals torch's FP32->BF16
    conversion (round to nearest even), including ties and subnormals."""
    torch = pytest.importorskip("torch")
    from _common import bf16_round
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(0, 3, 10000), rng.uniform(-1, 1, 1000) * 1e-39,
                        [1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(1.0 + 2.0 ** -8), 0.0, -0.0]]).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).float().numpy()
    assert np.array_equal(bf16_round(x).view(np.uint32), want.view(np.uint32))


# ---------------------------------------------------------------- the paper's visibility (Sec. 3.2)
def test_tri_visibility_lone_triangle_and_back_faces():
    # a lone triangle owns pixels from both sides: all three vertices visible;
    # with back faces culled it is invisible from its back side
    xp = np.array([[0.0, 0, 0], [0.3, 0, 0], [0, 0.3, 0]])
    faces = np.array([[0, 1, 2]], np.int32)
    dirs = np.zeros((32, 3))
    dirs[:16, 2] = 1.0
    dirs[16:, 2] = -1.0
    b = O.visibility_tri(xp, faces, _frames_for(dirs), [0.1, 0.1, 0], 1.0, 64)[:, 0]
    assert np.all(b == 0xFFFFFFFF)
    bc = O.visibility_tri(xp, faces, _frames_for(dirs), [0.1, 0.1, 0], 1.0, 64, cull_back=True)[:, 0]
    up = bc & 0xFFFF
    down = bc >> 16
    # the triangle is wound counter-clockwise seen from +z; which side is "front"
    # depends on the frame's handedness: exactly one side survives the cull
    assert (np.all(up == 0xFFFF) and np.all(down == 0)) or (np.all(up == 0) and np.all(down == 0xFFFF))


def test_tri_visibility_parallel_quads_and_ownership():
    # the near quad covers the far quad's overlap: far triangles there own no
    # pixel, so far vertices inside the overlap are invisible from above
    def quad(x0, x1, y0, y1, z, n):
        xs = np.linspace(x0, x1, n)
        ys = np.linspace(y0, y1, n)
        X, Y = np.meshgrid(xs, ys)
        v = np.stack([X.ravel(), Y.ravel(), np.full(X.size, z)], 1)
        f = []
        for j in range(n - 1):
            for i in range(n - 1):
                a = j * n + i
                f += [(a, a + 1, a + n), (a + 1, a + n + 1, a + n)]
        return v, np.array(f, np.int32)
    v1, f1 = quad(-0.5, 0.5, -0.5, 0.5, 0.2, 9)
    v2, f2 = quad(0.0, 1.0, -0.5, 0.5, -0.2, 9)
    xp = np.concatenate([v1, v2])
    faces = np.concatenate([f1, f2 + len(v1)])
    dirs = np.zeros((32, 3))
    dirs[:, 2] = 1.0
    bits, tri = O.visibility_tri(xp, faces, _frames_for(dirs), [0.25, 0, 0], 1.2, 128, want_tri=True)
    up = (bits[:, 0] & 1) != 0
    n1 = len(v1)
    assert np.all(up[:n1])
    # a far vertex is visible iff one of its triangles owns a pixel: those
    # triangles all lie beyond the near quad's edge x = 0.5 (step 0.125)
    far_x = v2[:, 0]
    assert np.all(~up[n1:][far_x < 0.5 - 0.13])
    assert np.all(up[n1:][far_x > 0.5 + 0.01])
    # every owning triangle index is a real triangle, and no far triangle owns a
    # pixel whose centre lies inside the near quad
    t0 = tri[0]
    assert t0.max() < len(faces) and t0.min() >= -1
    R, half, cx = 128, 1.2, 0.25
    jj, ii = np.nonzero(t0 >= len(f1))
    assert len(ii) > 0
    e1, e2, _ = _frames_for(dirs)[0].reshape(3, 3)
    s = (ii + 0.5) / R * 2 * half - half
    t = (jj + 0.5) / R * 2 * half - half
    wx = cx + s * e1[0] + t * e2[0]              # world x of the pixel centres the far quad owns
    wy = s * e1[1] + t * e2[1]
    assert np.all((wx > 0.5 - 2 * half / R) | (np.abs(wy) > 0.5 - 2 * half / R))


def test_tri_visibility_tied_triangles_all_appear():
    # two coincident triangles with distinct vertices lie at the same least
    # depth at every pixel: both appear, so all six vertices are visible; a
    # copy moved behind them appears nowhere
    base = np.array([[0.0, 0, 0], [0.4, 0, 0], [0, 0.4, 0]])
    behind = base - np.array([0, 0, 0.05])
    xp = np.concatenate([base, base, behind])
    faces = np.array([[3, 4, 5], [0, 1, 2], [6, 7, 8]], np.int32)
    dirs = np.zeros((32, 3))
    dirs[:, 2] = 1.0
    bits, tri = O.visibility_tri(xp, faces, _frames_for(dirs), [0.1, 0.1, 0], 1.0, 64, want_tri=True)
    assert np.all(bits[:6, 0] == 0xFFFFFFFF)
    assert np.all(bits[6:, 0] == 0)
    assert set(np.unique(tri[0])) == {-1, 0}     # the reported owner is the least tied index


def test_tri_visibility_convex_sphere_hemisphere():
    v, f, n = synth._tessellate_capsule((0, 0, 0), (0, 0, 0), 0.5, 600)
    dirs = synth.fibonacci_directions(128)
    bits = O.visibility_tri(v, f, _frames_for(dirs), [0, 0, 0], 0.6, 256)
    vb = np.unpackbits(bits.view(np.uint8), bitorder="little").reshape(len(v), -1)[:, :128]
    cosines = n @ dirs.T
    # front-facing triangles of a convex body are never hidden; a vertex whose
    # triangles all face away appears nowhere - except that a back triangle
    # reaching the silhouette may tie the front surface's integer depth at a
    # grazing pixel, so the back-side margin is wider than the front one
    assert np.all(vb[cosines >= 0.35] == 1)
    assert np.all(vb[cosines <= -0.5] == 0)


def test_vis_filters_match_numpy_median_and_mean():
    rng = np.random.default_rng(3)
    Nv, D, Kv = 300, 64, 19
    pts = rng.normal(size=(Nv, 3))
    knn_v = synth.knn_indices(pts, pts, Kv)
    V = (rng.random((Nv, D)) < 0.6).astype(np.uint8)
    bits = np.packbits(V, axis=1, bitorder="little").view(np.uint32)
    got = O.vis_filter(bits, knn_v)
    m1 = np.median(V[knn_v], axis=1)            # [Nv, D]: median over the Kv neighbours
    m2 = np.median(m1[knn_v], axis=1)
    mean = np.mean(m2[knn_v], axis=1)
    np.testing.assert_array_equal(got, np.rint(mean * Kv).astype(np.uint8))


def test_vis_filters_special_cases():
    rng = np.random.default_rng(4)
    Nv, Kv = 200, 19
    pts = rng.normal(size=(Nv, 3))
    knn_v = synth.knn_indices(pts, pts, Kv)
    ones = np.full((Nv, 1), 0xFFFFFFFF, np.uint32)
    assert np.all(O.vis_filter(ones, knn_v) == Kv)
    assert np.all(O.vis_filter(np.zeros_like(ones), knn_v) == 0)
    # a single visible vertex among invisible ones is noise: the medians remove it
    V = np.zeros((Nv, 32), np.uint8)
    V[17, :] = 1
    b = np.packbits(V, axis=1, bitorder="little").view(np.uint32)
    assert np.all(O.vis_filter(b, knn_v) == 0)
    with pytest.raises(ValueError):
        O.vis_filter(ones, knn_v[:, :18])        # even Kv has no unique binary median


def test_soft_shading_reduces_to_bits_for_saturated_counts():
    # counts of 0 or Kv are the hard bits: soft shading equals bit shading
    sc = synth.config_scene("c3_fd")
    av = sc.avatar
    sk = O.skin(av, O.fk(av.parents, av.joints, av.pose))
    rng = np.random.default_rng(5)
    D = sc.frames.shape[0]
    V = (rng.random((av.Nv, D)) < 0.7).astype(np.uint8)
    bits = np.packbits(V, axis=1, bitorder="little").view(np.uint32)
    args = (sk["xd"], sk["nd"], sk["ag"], sk["rg"], sk["pg"], sk["ubar"], av.knn)
    light = (sc.light.L, sc.light.A, sc.light.w, sc.dmap, sc.camera.center)
    c_bits, r_bits, _ = O.shade(*args, bits, *light, D)
    c_soft, r_soft, _ = O.shade_soft(*args, V * 19, 19, *light)
    np.testing.assert_allclose(r_soft, r_bits, rtol=1e-12, atol=1e-14)
    # and soft shading is linear in the counts: halving every count halves the
    # sums of lit, unculled Gaussians' radiance before gamma
    _, r_half, _ = O.shade_soft(*args, V * 10, 20, *light)
    np.testing.assert_allclose(r_half, 0.5 * r_bits, rtol=1e-12, atol=1e-14)


# ---------------------------------------------------------------- nearest neighbours
def test_knn_matches_scipy_and_breaks_ties_by_index():
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(9)
    ref = rng.normal(size=(400, 3)).astype(np.float32)
    x = rng.normal(size=(300, 3)).astype(np.float32)
    idx, d2 = O.knn(x, ref, 7, want_dist=True)
    dd, ii = cKDTree(ref.astype(np.float64)).query(x.astype(np.float64), k=7)
    np.testing.assert_allclose(np.sqrt(d2), dd, rtol=1e-12)          # the same distances as a k-d tree
    assert np.mean(idx == ii) > 0.999                                 # and the same points (no ties here)
    # exact ties (a lattice) go to the lower index; a point's own copy is first
    g = np.stack(np.meshgrid(np.arange(4), np.arange(4), np.arange(4), indexing="ij"), -1).reshape(-1, 3)
    q = np.array([[1.5, 1.5, 1.5]], np.float32)                       # 8 lattice points at equal distance
    k8 = O.knn(q, g, 8)[0]
    assert list(k8) == sorted(k8)
    assert np.allclose(np.linalg.norm(g[k8] - q, axis=1), np.sqrt(0.75))
    self_k = O.knn(g, g, 1)[:, 0]
    assert np.array_equal(self_k, np.arange(len(g)))


def test_knn_distances_follow_the_fp64_definition():
    # the squared distance is the FP64 value of (d0 d0 + d1 d1) + d2 d2 of the
    # FP32 coordinates: within 2 FP64 ulps of the exact rational value
    from fractions import Fraction
    rng = np.random.default_rng(10)
    ref = rng.uniform(-1, 1, size=(50, 3)).astype(np.float32)
    x = rng.uniform(-1, 1, size=(20, 3)).astype(np.float32)
    idx, d2 = O.knn(x, ref, 3, want_dist=True)
    for i in range(len(x)):
        for k in range(3):
            ex = sum((Fraction(float(x[i, c])) - Fraction(float(ref[idx[i, k], c]))) ** 2 for c in range(3))
            assert abs(Fraction(d2[i, k]) - ex) <= 2 * 2.0 ** -52 * ex
            dd = (x[i].astype(np.float64) - ref[idx[i, k]].astype(np.float64))
            assert d2[i, k] == (dd[0] * dd[0] + dd[1] * dd[1]) + dd[2] * dd[2]


# ---------------------------------------------------------------- image loss (Eq. 5)
def test_ssim_identity_symmetry_and_constant_images():
    from oracle import ssim as S
    rng = np.random.default_rng(12)
    x = rng.uniform(0, 1, size=(3, 40, 36))
    y = np.clip(x + rng.normal(0, 0.1, x.shape), 0, 1)
    np.testing.assert_allclose(S.ssim_map(x, x), 1.0, atol=1e-12)                 # SSIM(x, x) = 1
    np.testing.assert_allclose(S.ssim_map(x, y), S.ssim_map(y, x), atol=1e-14)   # symmetric
    assert S.ssim_map(x, y).mean() < 0.99
    # constant images a, b: away from the border the window sees only the
    # constant, so SSIM = (2ab + C1) / (a^2 + b^2 + C1) (zero variances)
    a, b = 0.3, 0.7
    s = S.ssim_map(np.full((1, 32, 32), a), np.full((1, 32, 32), b))
    inner = s[0, 5:-5, 5:-5]
    np.testing.assert_allclose(inner, (2 * a * b + S.C1) / (a * a + b * b + S.C1), rtol=1e-12)
    # the window is a normalised Gaussian of sigma 1.5
    g = S.gauss_1d()
    assert abs(g.sum() - 1) < 1e-15 and np.argmax(g) == 5
    np.testing.assert_allclose(g[4] / g[5], np.exp(-1 / (2 * 1.5 ** 2)), rtol=1e-14)


def test_ssim_of_a_constant_against_a_checkerboard():
    """x = a (constant), y = a + b (-1)^(i+j): with the normalised window's
    alternating sum A = sum_k (-1)^k g_k, at an interior pixel of parity p
    mu_y = a + b p A^2, sigma_y^2 = b^2 (1 - A^4), sigma_x = sigma_xy = 0, so
    SSIM = (2 a mu_y + C1) C2 / ((a^2 + mu_y^2 + C1)(sigma_y^2 + C2)) with
    C1 = 0.01^2 and C2 = 0.03^2 (the 3DGS constants, dynamic range 1)."""
    from oracle import ssim as S
    a, b, n = 0.5, 0.2, 40
    ii, jj = np.mgrid[0:n, 0:n]
    par = np.where((ii + jj) % 2 == 0, 1.0, -1.0)
    x = np.full((1, n, n), a)
    y = (a + b * par)[None]
    g = S.gauss_1d()
    A = np.sum(g * (-1.0) ** np.arange(len(g)))
    mu = a + b * par * A * A
    var = b * b * (1 - A ** 4)
    c1, c2 = 0.01 ** 2, 0.03 ** 2
    want = (2 * a * mu + c1) * c2 / ((a * a + mu * mu + c1) * (var + c2))
    np.testing.assert_allclose(S.ssim_map(x, y)[0, 6:-6, 6:-6], want[6:-6, 6:-6], rtol=1e-10)


def test_image_loss_weights_and_the_paper_lambda():
    """L_img = (1 - lambda) L1 + lambda (1 - SSIM): lambda = 0 gives the mean
    absolute error alone, lambda = 1 the D-SSIM alone, and the default is the
    paper's lambda_img (tests/golden/sec33_loss_weights.txt)."""
    import inspect
    from oracle import ssim as S
    rng = np.random.default_rng(14)
    x = rng.uniform(0, 1, size=(3, 24, 20))
    y = rng.uniform(0, 1, size=(3, 24, 20))
    assert abs(S.image_loss(x, y, 0.0) - np.abs(x - y).mean()) < 1e-15
    assert abs(S.image_loss(x, y, 1.0) - (1.0 - S.ssim_map(x, y).mean())) < 1e-15
    lam = golden_constants("sec33_loss_weights.txt")["lambda_img"]
    assert inspect.signature(S.image_loss).parameters["lam"].default == lam
    assert abs(S.image_loss(x, y) - ((1 - lam) * np.abs(x - y).mean() + lam * (1 - S.ssim_map(x, y).mean()))) < 1e-15


def test_image_loss_gradient_matches_finite_differences():
    from oracle import ssim as S
    rng = np.random.default_rng(13)
    x = rng.uniform(0, 1, size=(2, 14, 13))
    y = rng.uniform(0, 1, size=(2, 14, 13))
    loss, g = S.image_loss_grad(x, y, 0.2)
    assert abs(loss - S.image_loss(x, y, 0.2)) < 1e-14
    for (c, i, j) in [(0, 0, 0), (1, 7, 6), (0, 13, 12), (1, 3, 9)]:
        h = 1e-6
        xp, xm = x.copy(), x.copy()
        xp[c, i, j] += h
        xm[c, i, j] -= h
        fd = (S.image_loss(xp, y, 0.2) - S.image_loss(xm, y, 0.2)) / (2 * h)
        assert abs(fd - g[c, i, j]) < 1e-7 * max(1.0, abs(fd))


# ---------------------------------------------------------------- regularisers (Sec. 3.3)
def test_regularizers_closed_forms():
    from oracle import regularizers as RG
    xv = np.array([[0.0, 0, 0], [1.0, 0, 0], [3.0, 0, 0]])
    knn_v = np.array([[0, 1], [1, 0], [2, 1]])                 # each vertex and its nearest other vertex
    av = np.array([[0.2, 0.2, 0.2], [0.5, 0.1, 0.2], [0.5, 0.1, 0.9]])
    rv = np.array([0.3, 0.3, 0.6])
    pv = np.array([0.0, 1.0, 1.0])
    # smooth: pairs (0,1), (1,0), (2,1): |a| sums 0.4, 0.4, 0.7; |gamma| 0, 0, 0.3; |p| 1, 1, 0
    xg = np.array([[0.0, 0, 0], [1.0, 2.0, 0]])
    knn = np.array([[0], [1]])
    logscale = np.log(np.array([[0.004, 0.004, 0.004], [0.01, 0.002, 0.007]]))
    dxv = np.array([[0.0, 0, 0], [0.3, 0.4, 0], [0, 0, -2.0]])
    total, t, _ = RG.regularizers(xg, logscale, knn, xv, av, rv, pv, knn_v, dxv)
    assert abs(t["smooth"] - (0.4 + 0.4 + 0.7 + 0.3 + 2.0)) < 1e-12
    assert abs(t["mdist"] - 2.0) < 1e-12                       # Gaussian 0 sits on its vertex, Gaussian 1 at 2
    assert abs(t["disp"] - (0.5 + 2.0)) < 1e-12
    assert abs(t["scale"] - (0.005 + 0.002)) < 1e-12          # only 0.01 and 0.007 exceed s0 = 0.005
    w = RG.WEIGHTS
    assert abs(total - sum(w[k] * t[k] for k in t)) < 1e-12


def test_regularizer_weights_are_the_papers():
    """The weights and the scale threshold printed in Sec. 3.3
    (tests/golden/sec33_loss_weights.txt)."""
    from oracle import regularizers as RG
    gc = golden_constants("sec33_loss_weights.txt")
    assert RG.S0 == gc["s0"]
    assert RG.WEIGHTS == {k: gc["lambda_" + k] for k in ("smooth", "mdist", "disp", "scale")}


def test_regularizer_gradients_match_finite_differences():
    from oracle import regularizers as RG
    rng = np.random.default_rng(21)
    Nv, G = 30, 40
    xv = rng.normal(size=(Nv, 3))
    knn_v = synth.knn_indices(xv, xv, 5)
    xg = xv[rng.integers(0, Nv, G)] + 0.05 * rng.normal(size=(G, 3))
    knn = synth.knn_indices(xv, xg, 3)
    av, rv, pv = rng.uniform(size=(Nv, 3)), rng.uniform(size=Nv), rng.uniform(size=Nv)
    logscale = np.log(rng.uniform(0.001, 0.01, size=(G, 3)))
    dxv = 0.01 * rng.normal(size=(Nv, 3))
    args = dict(xg=xg, logscale=logscale, knn=knn, xv=xv, av=av, rv=rv, pv=pv, knn_v=knn_v, dxv=dxv)
    _, _, g = RG.regularizers(**args)
    for name, idx in (("xg", (3, 1)), ("logscale", (5, 2)), ("av", (7, 0)), ("rv", (2,)), ("pv", (11,)),
                      ("dxv", (4, 1))):
        h = 1e-7
        ap = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in args.items()}
        am = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in args.items()}
        ap[name][idx] += h
        am[name][idx] -= h
        fd = (RG.regularizers(**ap)[0] - RG.regularizers(**am)[0]) / (2 * h)
        assert abs(fd - g[name][idx]) < 1e-5 * max(1.0, abs(fd)), name


# ---------------------------------------------------------------- displacement MLP
def test_mlp_matches_torch_layers_and_closed_forms():
    from oracle import mlp as M
    w = synth.mlp_weights(1)
    rng = np.random.default_rng(31)
    x = rng.normal(0, 0.5, size=(50, 3))
    theta = rng.normal(0, 0.3, size=72)
    got = M.forward(x, theta, **w)
    # the same network from torch's own layers in FP64
    tw = {k: torch.tensor(v, dtype=torch.float64) for k, v in w.items()}
    p = 2 * math.pi * torch.tensor(x) @ tw["Bf"].T
    inp = torch.cat([torch.sin(p), torch.cos(p), torch.tensor(theta).expand(len(x), -1)], 1)
    net = torch.nn.Sequential(torch.nn.Linear(200, 256), torch.nn.ReLU(), torch.nn.Linear(256, 256),
                              torch.nn.ReLU(), torch.nn.Linear(256, 256), torch.nn.ReLU(),
                              torch.nn.Linear(256, 3)).double()
    with torch.no_grad():
        for lin, (W, b) in zip([net[0], net[2], net[4], net[6]], [("W1", "b1"), ("W2", "b2"), ("W3", "b3"),
                                                                  ("W4", "b4")]):
            lin.weight.copy_(tw[W])
            lin.bias.copy_(tw[b])
        want = net(inp).numpy()
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-15)
    # with the last layer zero the output is its bias
    w0 = dict(w, W4=np.zeros_like(w["W4"]))
    np.testing.assert_allclose(M.forward(x, theta, **w0), np.broadcast_to(w["b4"], (50, 3)), atol=0)
    # Fourier features: sin^2 + cos^2 = 1, and integer frequencies are 1-periodic
    g = M.features(x, w["Bf"])
    np.testing.assert_allclose(g[:, :64] ** 2 + g[:, 64:] ** 2, 1.0, atol=1e-14)
    Bi = np.rint(w["Bf"])
    np.testing.assert_allclose(M.features(x + np.array([1.0, 0, 0]), Bi), M.features(x, Bi), atol=1e-9)
    # the bfloat16 rounding of the kernel's operands: nearest, ties to even
    assert M.bf16(1 + 2.0 ** -8) == 1.0 and M.bf16(1 + 3 * 2.0 ** -8) == 1 + 2.0 ** -6


# ---------------------------------------------------------------- densification (App. B, Alg. 1)
def _torus(n, m, R=1.0, r=0.3):
    """A closed n x m torus grid, each quad split in two: every vertex has
    exactly six incident triangles (the valence Alg. 1 assumes)."""
    i, j = np.meshgrid(np.arange(n), np.arange(m), indexing="ij")
    th, ph = 2 * np.pi * i / n, 2 * np.pi * j / m
    xv = np.stack([(R + r * np.cos(ph)) * np.cos(th), (R + r * np.cos(ph)) * np.sin(th), r * np.sin(ph)], -1)
    idx = lambda a, b: (a % n) * m + (b % m)
    faces = []
    for a in range(n):
        for b in range(m):
            faces.append((idx(a, b), idx(a + 1, b), idx(a + 1, b + 1)))
            faces.append((idx(a, b), idx(a + 1, b + 1), idx(a, b + 1)))
    return xv.reshape(-1, 3), np.array(faces)


def test_densify_counts_and_densities():
    from oracle import densify as DN
    xv, faces = _torus(12, 10)
    nv = xv.shape[0]
    rng = np.random.default_rng(41)
    G, Kg = 700, 3
    knn = np.stack([rng.choice(nv, Kg, replace=False) for _ in range(G)])
    rand = rng.integers(0, 2 ** 32, size=(4000, 3), dtype=np.uint64)
    out = DN.densify(knn, faces, xv, rand)
    # D_v equals numpy's bincount of the neighbour lists
    np.testing.assert_array_equal(out["Dv"], np.bincount(knn.ravel(), minlength=nv))
    # valence 6 everywhere: the triangle densities sum to the number of Gaussians
    assert abs(out["df"].sum() - G) < 1e-9
    # P, N' and the weights against exact rationals
    from fractions import Fraction
    P = [max(Fraction(0), Fraction(1) - Fraction(int(s), 6 * Kg))
         for s in out["Dv"][faces].sum(1)]
    assert all(Fraction(int(w), 6 * Kg) == p for w, p in zip(out["w"], P))
    assert out["n_new"] == int(Fraction(0.02) * sum(P) // 1)
    assert out["ng"].sum() == out["n_new"] and np.all(out["ng"][out["w"] == 0] == 0)


def test_densify_uniform_and_saturated_meshes():
    from oracle import densify as DN
    xv, faces = _torus(8, 8)
    nv, Kg = xv.shape[0], 4
    rand = np.random.default_rng(3).integers(0, 2 ** 32, size=(2000, 3), dtype=np.uint64)
    # every vertex in S_g of exactly c Gaussians: d_f = 3c / (6 K_g) on every triangle
    for c in (1, 3, 8):
        knn = np.stack([np.roll(np.repeat(np.arange(nv), c), -k * c) for k in range(Kg)], 1)  # each vertex c K_g times
        out = DN.densify(knn, faces, xv, rand)
        assert np.all(out["Dv"] == c * Kg)
        np.testing.assert_allclose(out["df"], 3 * c * Kg / (6 * Kg))
        want = int(np.floor(0.02 * faces.shape[0] * max(0.0, 1.0 - 0.5 * c)))
        assert out["n_new"] == want
    # saturated (d_f >= d0 everywhere): nothing is added
    assert DN.densify(knn, faces, xv, rand)["n_new"] == 0


def test_densify_sampling_follows_the_weights():
    from oracle import densify as DN
    xv, faces = _torus(6, 6)
    nv, Kg = xv.shape[0], 2
    # a single uncovered triangle's vertices: all other vertices saturated
    hole = faces[5]
    others = np.setdiff1d(np.arange(nv), hole)
    knn = np.repeat(others, 12)[:, None].repeat(Kg, 1)
    rand = np.random.default_rng(8).integers(0, 2 ** 32, size=(20000, 3), dtype=np.uint64)
    out = DN.densify(knn, faces, xv, rand, p0=50.0)
    # only triangles touching no covered vertex (the hole's own) get draws
    assert out["n_new"] > 0 and set(out["tri"]) <= set(np.flatnonzero(out["w"] > 0))
    # the empirical frequencies match w / W (a chi-square bound at p ~ 1e-6)
    out = DN.densify(np.arange(nv)[:, None].repeat(Kg, 1)[: nv // 2], faces, xv, rand, p0=200.0)
    w, n = out["w"].astype(float), out["n_new"]
    exp = n * w / w.sum()
    m = exp > 0
    chi2 = ((out["ng"][m] - exp[m]) ** 2 / exp[m]).sum()
    dof = m.sum() - 1
    assert np.all(out["ng"][~m] == 0) and chi2 < dof + 7 * np.sqrt(2 * dof)


def test_densify_places_points_uniformly_on_the_triangle():
    from oracle import densify as DN
    xv = np.array([[0.0, 0, 0], [1.0, 0, 0], [0.0, 2.0, 0], [5.0, 5.0, 5.0]])
    faces = np.array([[0, 1, 2], [1, 3, 2]])
    knn = np.full((6, 1), 3)  # vertex 3 saturates face 1 (S = 6 = 6 K_g): face 0 gets every draw
    rand = np.random.default_rng(12).integers(0, 2 ** 32, size=(30000, 3), dtype=np.uint64)
    out = DN.densify(knn, faces, xv, rand, d0=1.0, p0=20000.0)
    x = out["x"]
    assert np.all(out["tri"] == 0) and len(x) > 10000
    # barycentrics of the right triangle (0,0) (1,0) (0,2): u = x, v = y / 2, inside
    u, v = x[:, 0], x[:, 1] / 2
    assert np.all(u >= 0) and np.all(v >= 0) and np.all(u + v <= 1) and np.all(x[:, 2] == 0)
    # uniform on the triangle: mean = centroid, and each half of the area gets half
    np.testing.assert_allclose(x.mean(0), [1 / 3, 2 / 3, 0], atol=0.01)
    assert abs((u + v < np.sqrt(0.5)).mean() - 0.5) < 0.01


# ---------------------------------------------------------------- Adam
def test_adam_matches_torch_and_closed_forms():
    from oracle import adam as AD
    rng = np.random.default_rng(51)
    p0 = rng.normal(size=300)
    gs = [rng.normal(size=300) * 10.0 ** rng.uniform(-3, 1) for _ in range(6)]
    # torch.optim.Adam in FP64, same hyper-parameters
    tp = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=0.01, betas=(0.9, 0.999), eps=1e-15)
    p, m, v = p0.copy(), np.zeros(300), np.zeros(300)
    for t, g in enumerate(gs, 1):
        tp.grad = torch.tensor(g)
        opt.step()
        p, m, v = AD.step(p, g, m, v, t, 0.01)
        np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-13, atol=1e-15)
    # first step: m_hat = g, v_hat = g^2, so the step is lr g / (|g| + eps), about lr sign(g)
    g = rng.normal(size=50)
    p1, _, _ = AD.step(np.zeros(50), g, np.zeros(50), np.zeros(50), 1, 0.003)
    np.testing.assert_allclose(p1, -0.003 * g / (np.abs(g) + 1e-15), rtol=1e-13)
    # a constant gradient keeps that step for every t (the bias corrections cancel)
    p, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    g = np.array([2.0, -0.5, 1e-3, -7.0])
    for t in range(1, 30):
        q, m, v = AD.step(p, g, m, v, t, 0.1)
        np.testing.assert_allclose(q - p, -0.1 * g / (np.abs(g) + 1e-15), rtol=1e-10)
        p = q
    # bfloat16 storage: the result is a bfloat16 value nearest to the FP64 update
    # (1 - 3 2^-9 lies halfway between 1 - 2^-7 and 1 - 2^-8: ties to the even 1 - 2^-7;
    #  1 + 3 2^-9 is nearer 1 + 2^-7 than 1)
    pb, _, _ = AD.step(np.full(3, 1.0), np.array([1.0, -1.0, 0.0]), np.zeros(3), np.zeros(3), 1, 3 * 2.0 ** -9,
                       bf16=True)
    np.testing.assert_array_equal(pb, [1.0 - 2.0 ** -7, 1.0 + 2.0 ** -7, 1.0])
