"""Seeded synthetic avatars shaped like the workloads of "Interactive Rendering
of Relightable and Animatable Gaussian Avatars" (arXiv 2407.10707).

This module only PRODUCES INPUTS.  It holds none of the render path's
arithmetic (no skinning, no rasterisation, no shading, no splatting); both the
CUDA path and the FP64 oracle consume what it returns.

What stands in for the paper's data (Sec. 3.1, Sec. 3.5, Sec. 4.1):
  * the SDF-extracted, remeshed canonical body mesh (about 40K vertices)
    -> a union of 16 closed capsules around a 24-joint SMPL-shaped skeleton,
       tessellated to a requested vertex count;
  * vertex attributes: albedo U(0.2,0.9)^3, roughness U(0.3,0.9), specular
    tint U(0,1), analytic capsule normals, dense 24-joint LBS weights
    (softmax of -dist^2/sigma^2 to the bone segments), displacement 0;
  * Gaussians sampled uniformly by area on the surface with log-scales
    N(-4,0.3), uniform unit quaternions, opacity U(0.3,0.95); their K nearest
    vertices (the set S_g of Eq. 1) by brute-force-equivalent KD-tree search;
  * pose: random joint rotations within +-30 degrees;
  * a lat-long environment light with log-normal radiance (ln L ~ N(-1,0.5)),
    texel-centre directions and exact band solid angles;
  * D visibility viewpoints on a Fibonacci sphere with orthonormal frames, and
    the map d(k) from light texel k to its nearest viewpoint;
  * a pinhole camera framing the body at about 80% of the image height.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# SMPL-shaped 24-joint kinematic tree (joint j rotates the bone that starts at j).
PARENTS = np.array([-1, 0, 0, 0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 9, 9, 12, 13, 14,
                    16, 17, 18, 19, 20, 21], dtype=np.int32)

# Rest (T-pose) joint positions in metres, y up, pelvis at the origin.
REST_JOINTS = np.array([
    [0.00, 0.00, 0.00],    # 0 pelvis
    [0.09, -0.08, 0.00],   # 1 L hip
    [-0.09, -0.08, 0.00],  # 2 R hip
    [0.00, 0.11, 0.00],    # 3 spine1
    [0.10, -0.48, 0.00],   # 4 L knee
    [-0.10, -0.48, 0.00],  # 5 R knee
    [0.00, 0.24, 0.00],    # 6 spine2
    [0.10, -0.88, 0.00],   # 7 L ankle
    [-0.10, -0.88, 0.00],  # 8 R ankle
    [0.00, 0.30, 0.00],    # 9 spine3
    [0.10, -0.93, 0.12],   # 10 L foot
    [-0.10, -0.93, 0.12],  # 11 R foot
    [0.00, 0.50, 0.00],    # 12 neck
    [0.07, 0.42, 0.00],    # 13 L collar
    [-0.07, 0.42, 0.00],   # 14 R collar
    [0.00, 0.58, 0.00],    # 15 head
    [0.17, 0.44, 0.00],    # 16 L shoulder
    [-0.17, 0.44, 0.00],   # 17 R shoulder
    [0.43, 0.44, 0.00],    # 18 L elbow
    [-0.43, 0.44, 0.00],   # 19 R elbow
    [0.68, 0.44, 0.00],    # 20 L wrist
    [-0.68, 0.44, 0.00],   # 21 R wrist
    [0.76, 0.44, 0.00],    # 22 L hand
    [-0.76, 0.44, 0.00],   # 23 R hand
], dtype=np.float64)

# Capsules (endpoint a, endpoint b, radius) making up the body surface.
CAPSULES = [
    ((0.00, -0.05, 0.00), (0.00, 0.38, 0.00), 0.150),   # torso
    ((-0.17, 0.43, 0.00), (0.17, 0.43, 0.00), 0.060),   # shoulders
    ((0.00, 0.42, 0.00), (0.00, 0.56, 0.00), 0.050),    # neck
    ((0.00, 0.64, 0.01), (0.00, 0.68, 0.01), 0.100),    # head
    ((0.09, -0.08, 0.00), (0.10, -0.48, 0.00), 0.075),  # L thigh
    ((-0.09, -0.08, 0.00), (-0.10, -0.48, 0.00), 0.075),
    ((0.10, -0.48, 0.00), (0.10, -0.88, 0.00), 0.052),  # L shin
    ((-0.10, -0.48, 0.00), (-0.10, -0.88, 0.00), 0.052),
    ((0.10, -0.90, -0.02), (0.10, -0.92, 0.14), 0.040),  # L foot
    ((-0.10, -0.90, -0.02), (-0.10, -0.92, 0.14), 0.040),
    ((0.17, 0.44, 0.00), (0.43, 0.44, 0.00), 0.046),    # L upper arm
    ((-0.17, 0.44, 0.00), (-0.43, 0.44, 0.00), 0.046),
    ((0.43, 0.44, 0.00), (0.68, 0.44, 0.00), 0.038),    # L forearm
    ((-0.43, 0.44, 0.00), (-0.68, 0.44, 0.00), 0.038),
    ((0.68, 0.44, 0.00), (0.80, 0.44, 0.00), 0.030),    # L hand
    ((-0.68, 0.44, 0.00), (-0.80, 0.44, 0.00), 0.030),
]


def _capsule_area(a, b, r):
    length = float(np.linalg.norm(np.subtract(b, a)))
    return 2.0 * math.pi * r * length + 4.0 * math.pi * r * r


def _orthonormal_pair(axis):
    axis = axis / np.linalg.norm(axis)
    helper = np.array([1.0, 0.0, 0.0]) if abs(axis[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    u = np.cross(axis, helper)
    u /= np.linalg.norm(u)
    v = np.cross(axis, u)
    return u, v


def _tessellate_capsule(a, b, r, n_vert):
    """Closed genus-0 capsule mesh with about n_vert vertices, outward winding.

    Returns vertices [n,3], faces [f,3] (local indices) and analytic normals.
    """
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    axis = b - a
    length = float(np.linalg.norm(axis))
    if length < 1e-9:
        axis = np.array([0.0, 1.0, 0.0])
        length = 0.0
    else:
        axis = axis / length
    u, v = _orthonormal_pair(axis)
    unrolled = length + math.pi * r
    segs = max(6, int(round(math.sqrt(max(n_vert - 2, 12) * 2.0 * math.pi * r / unrolled))))
    rings = max(2, int(round((n_vert - 2) / segs)))
    verts = []
    normals = []
    # pole at a
    verts.append(a - r * axis)
    normals.append(-axis)
    for i in range(rings):
        s = (i + 1) * unrolled / (rings + 1)
        if s < 0.5 * math.pi * r:
            phi = s / r                      # angle from the pole at a
            axial = -r * math.cos(phi)
            rad = r * math.sin(phi)
            base = a
            n_ax = -math.cos(phi)
        elif s < 0.5 * math.pi * r + length:
            axial = s - 0.5 * math.pi * r
            rad = r
            base = a
            n_ax = 0.0
        else:
            phi = (s - 0.5 * math.pi * r - length) / r   # angle from the equator at b
            axial = r * math.sin(phi)
            rad = r * math.cos(phi)
            base = b
            n_ax = math.sin(phi)
        n_rad = math.sqrt(max(0.0, 1.0 - n_ax * n_ax))
        for j in range(segs):
            ang = 2.0 * math.pi * (j + 0.5 * (i % 2)) / segs
            d = math.cos(ang) * u + math.sin(ang) * v
            verts.append(base + axial * axis + rad * d)
            normals.append(n_ax * axis + n_rad * d)
    verts.append(b + r * axis)
    normals.append(axis)
    verts = np.array(verts)
    normals = np.array(normals)
    faces = []
    first = 1
    # fan around the pole at a
    for j in range(segs):
        faces.append((0, first + (j + 1) % segs, first + j))
    for i in range(rings - 1):
        r0 = first + i * segs
        r1 = first + (i + 1) * segs
        for j in range(segs):
            j1 = (j + 1) % segs
            faces.append((r0 + j, r0 + j1, r1 + j))
            faces.append((r0 + j1, r1 + j1, r1 + j))
    last = first + (rings - 1) * segs
    pole_b = len(verts) - 1
    for j in range(segs):
        faces.append((pole_b, last + j, last + (j + 1) % segs))
    faces = np.array(faces, dtype=np.int64)
    # make the winding outward (checked against the analytic normal)
    p0, p1, p2 = verts[faces[:, 0]], verts[faces[:, 1]], verts[faces[:, 2]]
    fn = np.cross(p1 - p0, p2 - p0)
    outward = np.einsum("ij,ij->i", fn, normals[faces].mean(axis=1)) >= 0
    faces[~outward] = faces[~outward][:, [0, 2, 1]]
    return verts, faces, normals


def _bone_segments():
    """Segment of each joint's bone: from the joint to the mean of its children
    (leaves extend 8 cm away from the parent)."""
    segs = np.zeros((24, 2, 3))
    for j in range(24):
        children = np.where(PARENTS == j)[0]
        start = REST_JOINTS[j]
        if len(children):
            end = REST_JOINTS[children].mean(axis=0)
        else:
            d = REST_JOINTS[j] - REST_JOINTS[PARENTS[j]]
            end = start + 0.08 * d / max(np.linalg.norm(d), 1e-9)
        segs[j, 0], segs[j, 1] = start, end
    return segs


def _point_segment_dist2(p, a, b):
    ab = b - a
    t = np.clip(((p - a) @ ab) / max(ab @ ab, 1e-12), 0.0, 1.0)
    q = a + t[:, None] * ab
    return np.sum((p - q) ** 2, axis=1)


@dataclass
class Avatar:
    """Canonical avatar (mesh M, Gaussians G) plus per-frame inputs."""
    # mesh
    xv: np.ndarray          # [Nv,3] canonical vertex positions
    faces: np.ndarray       # [F,3] int32
    nv: np.ndarray          # [Nv,3] unit normals
    wv: np.ndarray          # [Nv,24] LBS weights (rows sum to 1)
    av: np.ndarray          # [Nv,3] albedo
    rv: np.ndarray          # [Nv] roughness
    pv: np.ndarray          # [Nv] specular tint
    dxv: np.ndarray         # [Nv,3] displacement
    # Gaussians
    xg: np.ndarray          # [G,3]
    logscale: np.ndarray    # [G,3]
    quat: np.ndarray        # [G,4] (w,x,y,z) unit
    opacity: np.ndarray     # [G]
    knn: np.ndarray         # [G,K] int32
    # skeleton / pose
    parents: np.ndarray = field(default_factory=lambda: PARENTS.copy())
    joints: np.ndarray = field(default_factory=lambda: REST_JOINTS.copy())
    pose: np.ndarray = None  # [24,3] axis-angle

    @property
    def G(self):
        return self.xg.shape[0]

    @property
    def Nv(self):
        return self.xv.shape[0]

    @property
    def F(self):
        return self.faces.shape[0]

    @property
    def K(self):
        return self.knn.shape[1]


def body_mesh(n_vertices: int):
    """Capsule-union body surface with about n_vertices vertices."""
    areas = np.array([_capsule_area(*c) for c in CAPSULES])
    share = areas / areas.sum()
    vs, fs, ns = [], [], []
    off = 0
    for (a, b, r), s in zip(CAPSULES, share):
        v, f, n = _tessellate_capsule(a, b, r, max(14, int(round(s * n_vertices))))
        vs.append(v)
        fs.append(f + off)
        ns.append(n)
        off += len(v)
    return (np.concatenate(vs), np.concatenate(fs).astype(np.int32),
            np.concatenate(ns))


def lbs_weights(xv: np.ndarray, sigma: float = 0.06) -> np.ndarray:
    segs = _bone_segments()
    d2 = np.stack([_point_segment_dist2(xv, segs[j, 0], segs[j, 1]) for j in range(24)], axis=1)
    logits = -d2 / (sigma * sigma)
    logits -= logits.max(axis=1, keepdims=True)
    w = np.exp(logits)
    w /= w.sum(axis=1, keepdims=True)
    return w


def sample_surface(rng, xv, faces, n):
    p0, p1, p2 = xv[faces[:, 0]], xv[faces[:, 1]], xv[faces[:, 2]]
    area = 0.5 * np.linalg.norm(np.cross(p1 - p0, p2 - p0), axis=1)
    tri = rng.choice(len(faces), size=n, p=area / area.sum())
    r1 = np.sqrt(rng.random(n))
    r2 = rng.random(n)
    b0, b1, b2 = 1 - r1, r1 * (1 - r2), r1 * r2
    return b0[:, None] * p0[tri] + b1[:, None] * p1[tri] + b2[:, None] * p2[tri]


def knn_indices(xv: np.ndarray, pts: np.ndarray, k: int) -> np.ndarray:
    """Indices of the k nearest vertices (ascending distance) of each point."""
    from scipy.spatial import cKDTree
    _, idx = cKDTree(xv).query(pts, k=k)
    idx = np.asarray(idx).reshape(len(pts), k)
    return idx.astype(np.int32)


def vertex_knn(xv: np.ndarray, k: int = 19) -> np.ndarray:
    """The k nearest vertices of every vertex (itself first): the neighbourhoods
    of the visibility filters (K_v = 19 in the paper's experiments)."""
    return knn_indices(xv, xv, k)


def random_pose(rng, max_deg: float = 30.0) -> np.ndarray:
    axis = rng.normal(size=(24, 3))
    axis /= np.linalg.norm(axis, axis=1, keepdims=True)
    ang = np.deg2rad(rng.uniform(-max_deg, max_deg, size=(24, 1)))
    return axis * ang


def make_avatar(n_vertices: int, n_gaussians: int, seed: int, k: int = 4,
                pose_deg: float = 30.0, displacement: float = 0.0) -> Avatar:
    rng = np.random.default_rng(seed)
    xv, faces, nv = body_mesh(n_vertices)
    nvtx = len(xv)
    wv = lbs_weights(xv)
    av = rng.uniform(0.2, 0.9, size=(nvtx, 3))
    rv = rng.uniform(0.3, 0.9, size=nvtx)
    pv = rng.uniform(0.0, 1.0, size=nvtx)
    dxv = displacement * rng.normal(size=(nvtx, 3)) if displacement else np.zeros((nvtx, 3))
    xg = sample_surface(rng, xv, faces, n_gaussians)
    logscale = rng.normal(-4.0, 0.3, size=(n_gaussians, 3))
    q = rng.normal(size=(n_gaussians, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    opacity = rng.uniform(0.3, 0.95, size=n_gaussians)
    knn = knn_indices(xv, xg, k)
    pose = random_pose(rng, pose_deg)
    return Avatar(xv=xv, faces=faces, nv=nv, wv=wv, av=av, rv=rv, pv=pv, dxv=dxv,
                  xg=xg, logscale=logscale, quat=q, opacity=opacity, knn=knn,
                  pose=pose)


# ---------------------------------------------------------------------------
# Light, viewpoints, camera
# ---------------------------------------------------------------------------
@dataclass
class Light:
    L: np.ndarray    # [K,3] radiance
    A: np.ndarray    # [K] solid angle of each texel
    w: np.ndarray    # [K,3] unit direction towards the light
    rows: int = 0    # lat-long grid shape (0: not a grid)
    cols: int = 0


def latlong_light(rng, rows: int, cols: int, mu: float = -1.0, sd: float = 0.5) -> Light:
    """Texel (i,j): theta=(i+1/2)pi/rows from +y, phi=(j+1/2)2pi/cols,
    w=(sin t sin p, cos t, sin t cos p); A = exact band solid angle."""
    i = np.arange(rows)
    j = np.arange(cols)
    th = (i + 0.5) * math.pi / rows
    ph = (j + 0.5) * 2.0 * math.pi / cols
    T, P = np.meshgrid(th, ph, indexing="ij")
    w = np.stack([np.sin(T) * np.sin(P), np.cos(T), np.sin(T) * np.cos(P)], axis=-1).reshape(-1, 3)
    band = (np.cos(i * math.pi / rows) - np.cos((i + 1) * math.pi / rows)) * 2.0 * math.pi / cols
    A = np.repeat(band, cols)
    L = np.exp(rng.normal(mu, sd, size=(rows * cols, 3)))
    return Light(L=L, A=A, w=w, rows=rows, cols=cols)


def latlong_patch_order(rows: int, cols: int, pr: int = 4, pc: int = 8) -> np.ndarray:
    """A storage order of a rows x cols lat-long light grid (row-major texel
    index) that lists the texels patch by patch, pr rows by pc columns per
    patch (32 texels: one 32-light chunk of the shading kernels), patches in
    row-major order; the identity when the grid does not split into patches."""
    if rows <= 0 or cols <= 0 or rows % pr or cols % pc:
        return np.arange(max(rows * cols, 0), dtype=np.int32)
    idx = np.arange(rows * cols).reshape(rows // pr, pr, cols // pc, pc)
    return np.ascontiguousarray(idx.transpose(0, 2, 1, 3)).reshape(-1).astype(np.int32)


def permute_lights(scene, order):
    """The scene with light texel s taken from texel order[s] (radiance,
    solid angle, direction, and the viewpoint d(k) of each texel); a storage
    order of the same light."""
    import dataclasses
    o = np.asarray(order)
    lt = scene.light
    light = dataclasses.replace(lt, L=lt.L[o], A=lt.A[o], w=lt.w[o], rows=0, cols=0)
    return dataclasses.replace(scene, light=light, dmap=np.asarray(scene.dmap)[o])


def fibonacci_directions(n: int) -> np.ndarray:
    i = np.arange(n)
    z = 1.0 - (2.0 * i + 1.0) / n
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    rxy = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([rxy * np.cos(phi), rxy * np.sin(phi), z], axis=1)


def direction_frames(dirs: np.ndarray) -> np.ndarray:
    """Orthonormal frames [D,3,3]: rows e1, e2, w with w the given direction."""
    out = np.zeros((len(dirs), 3, 3))
    for d, w in enumerate(dirs):
        w = w / np.linalg.norm(w)
        e1, e2 = _orthonormal_pair(w)
        out[d, 0], out[d, 1], out[d, 2] = e1, e2, w
    return out


def nearest_viewpoint(light_w: np.ndarray, view_dirs: np.ndarray) -> np.ndarray:
    """d(k): index of the viewpoint with the largest dot product (ties -> lower)."""
    dots = light_w @ view_dirs.T
    return np.argmax(dots, axis=1).astype(np.int32)


@dataclass
class Camera:
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    R: np.ndarray        # [3,3] world-to-camera rotation
    t: np.ndarray        # [3] world-to-camera translation
    center: np.ndarray   # [3] camera centre in world space (= -R^T t)


def look_at_camera(width: int, height: int, eye, target=(0.0, -0.1, 0.0),
                   body_height: float = 1.75, fill: float = 0.8) -> Camera:
    eye = np.asarray(eye, np.float64)
    target = np.asarray(target, np.float64)
    fwd = target - eye
    dist = np.linalg.norm(fwd)
    fwd /= dist
    up = np.array([0.0, 1.0, 0.0])
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd])          # camera x right, y down, z forward
    t = -R @ eye
    f = fill * height * dist / body_height
    return Camera(fx=f, fy=f, cx=width / 2.0, cy=height / 2.0, width=width, height=height,
                  R=R, t=t, center=eye.copy())


# ---------------------------------------------------------------------------
# Workload presets (sizes of the paper-shaped configurations)
# ---------------------------------------------------------------------------
@dataclass
class Scene:
    avatar: Avatar
    light: Light
    view_dirs: np.ndarray   # [D,3]
    frames: np.ndarray      # [D,3,3]
    dmap: np.ndarray        # [K] int32
    camera: Camera
    depth_res: int
    window_center: np.ndarray  # [3]
    window_half: float
    vis_bias: float            # world units


def make_scene(n_vertices, n_gaussians, light_rows, light_cols, n_dirs, depth_res,
               width, height, seed, k=4, pose_deg=30.0, view_dirs=None,
               displacement=0.0, eye=(0.35, 0.05, 3.2)) -> Scene:
    av = make_avatar(n_vertices, n_gaussians, seed, k=k, pose_deg=pose_deg,
                     displacement=displacement)
    rng = np.random.default_rng(seed + 1000)
    light = latlong_light(rng, light_rows, light_cols)
    if view_dirs is None:
        view_dirs = fibonacci_directions(n_dirs)
    frames = direction_frames(view_dirs)
    dmap = nearest_viewpoint(light.w, view_dirs)
    cam = look_at_camera(width, height, eye)
    # the posed body stays inside the canonical reach of the skeleton from the
    # pelvis; the window is that sphere with a 25% margin.
    reach = float(np.max(np.linalg.norm(av.xv - av.joints[0], axis=1)))
    half = 1.25 * reach
    bias = 2.0 * (2.0 * half / depth_res)
    return Scene(avatar=av, light=light, view_dirs=view_dirs, frames=frames, dmap=dmap,
                 camera=cam, depth_res=depth_res, window_center=av.joints[0].copy(),
                 window_half=half, vis_bias=bias)


# Paper-shaped configurations: (Nv, G, light rows, light cols, D, depth res, W, H, seed)
def permute_gaussians(scene: Scene, order) -> Scene:
    """The scene with Gaussian i taken from Gaussian order[i] (positions,
    log-scales, rotations, opacities and neighbour lists); everything else as
    is.  A storage order, not a change of the avatar."""
    import dataclasses
    o = np.asarray(order)
    av = scene.avatar
    av2 = dataclasses.replace(av, xg=av.xg[o], logscale=av.logscale[o], quat=av.quat[o], opacity=av.opacity[o],
                              knn=av.knn[o])
    return dataclasses.replace(scene, avatar=av2)


def _hilbert_index(x: np.ndarray, y: np.ndarray, n: int) -> np.ndarray:
    """Index along the Hilbert curve of cells (x, y) of an n x n grid (n a power
    of two): consecutive indices are neighbouring cells."""
    x = np.array(x, np.int64)
    y = np.array(y, np.int64)
    d = np.zeros_like(x)
    s = n // 2
    while s > 0:
        rx = (x & s) > 0
        ry = (y & s) > 0
        d += s * s * ((3 * rx.astype(np.int64)) ^ ry.astype(np.int64))
        turn = ~ry                                       # rotate the quadrant into the curve's frame
        flip = turn & rx
        x[flip] = s - 1 - x[flip]
        y[flip] = s - 1 - y[flip]
        x[turn], y[turn] = y[turn].copy(), x[turn].copy()
        s //= 2
    return d


def face_normal_order(xv: np.ndarray, faces: np.ndarray, chunk: int = 1024, bins: int = 32) -> np.ndarray:
    """A storage order of a mesh's faces for the visibility raster: within
    each run of `chunk` faces (the raster's chunk, so every chunk keeps its
    faces and vertex range) the faces are listed stably by the position of
    their canonical normal's cell (bins x bins, octahedral map) along a
    Hilbert curve.  A warp's 32 faces then face nearly the same way, so
    toward most lights they are all back faces (left at the orientation
    test) or mostly front faces; the bits do not depend on the order."""
    xv = np.asarray(xv, np.float64)
    f = np.asarray(faces, np.int64)
    n = np.cross(xv[f[:, 1]] - xv[f[:, 0]], xv[f[:, 2]] - xv[f[:, 0]])
    n = n / np.maximum(np.linalg.norm(n, axis=1, keepdims=True), 1e-300)
    p = n[:, :2] / np.maximum(np.abs(n).sum(1, keepdims=True), 1e-300)
    q = p.copy()
    lower = n[:, 2] < 0                                   # fold the lower hemisphere (octahedral map)
    q[lower] = (1.0 - np.abs(p[lower][:, ::-1])) * np.where(p[lower] >= 0, 1.0, -1.0)
    cell = np.clip(np.floor((q + 1.0) * 0.5 * bins), 0, bins - 1).astype(np.int64)
    key = _hilbert_index(cell[:, 0], cell[:, 1], bins)
    order = np.arange(len(f), dtype=np.int64)
    for c in range(0, len(f), chunk):
        idx = order[c:c + chunk]
        order[c:c + chunk] = idx[np.argsort(key[c:c + chunk], kind="stable")]
    return order.astype(np.int32)


def permute_faces(scene: Scene, order) -> Scene:
    """The scene with face s taken from face order[s] (a storage order of
    the same mesh)."""
    import dataclasses
    av = dataclasses.replace(scene.avatar, faces=np.asarray(scene.avatar.faces)[np.asarray(order)])
    return dataclasses.replace(scene, avatar=av)


def nearest_vertex_order(scene: Scene) -> np.ndarray:
    """Stable order of the Gaussians by their nearest vertex (knn column 0)."""
    return np.argsort(scene.avatar.knn[:, 0], kind="stable").astype(np.int32)


CONFIGS = {
    "c1_small": dict(n_vertices=2562, n_gaussians=10_000, light_rows=8, light_cols=16,
                     n_dirs=64, depth_res=64, width=256, height=256, seed=0),
    "c2_paper": dict(n_vertices=50_000, n_gaussians=200_000, light_rows=16, light_cols=32,
                     n_dirs=512, depth_res=256, width=1024, height=1024, seed=1),
    "c3_fd": dict(n_vertices=2562, n_gaussians=1_000, light_rows=8, light_cols=16,
                  n_dirs=64, depth_res=64, width=64, height=64, seed=1),
    "c5_stress": dict(n_vertices=200_000, n_gaussians=1_000_000, light_rows=32, light_cols=64,
                      n_dirs=1024, depth_res=512, width=2048, height=2048, seed=3),
}


def config_scene(name: str, **overrides) -> Scene:
    kw = dict(CONFIGS[name])
    kw.update(overrides)
    return make_scene(**kw)


# ---------------------------------------------------------------------------
# Batched workloads: poses x cameras of mixed resolution, one light per pose
# ---------------------------------------------------------------------------
@dataclass
class Batch:
    scene: Scene            # the avatar, light texel geometry and visibility geometry
    poses: np.ndarray       # [B,24,3] axis-angle (pose 0 is the scene's own pose)
    lights: np.ndarray      # [B,K,3] radiance of each pose's environment light
    cameras: list           # [V] Camera
    view_pose: np.ndarray   # [V] int32, pose shown by each view

    @property
    def B(self):
        return self.poses.shape[0]

    @property
    def V(self):
        return len(self.cameras)


def make_batch(scene: Scene, n_poses: int, cams_per_pose: int, resolutions, seed: int,
               pose_deg: float = 30.0, dist: float = 3.2) -> Batch:
    """Pose p (random joint rotations within +-pose_deg; pose 0 = the scene's)
    lit by its own log-normal light, seen by cams_per_pose cameras orbiting
    the body at distance dist; resolutions (width, height) cycle over the views."""
    rng = np.random.default_rng(seed + 2000)
    poses = [scene.avatar.pose] + [random_pose(rng, pose_deg) for _ in range(n_poses - 1)]
    lights = [scene.light.L] + [np.exp(rng.normal(-1.0, 0.5, size=scene.light.L.shape))
                                for _ in range(n_poses - 1)]
    cams, vp = [], []
    v = 0
    for p in range(n_poses):
        az0 = rng.uniform(0.0, 2.0 * math.pi)
        for c in range(cams_per_pose):
            az = az0 + 2.0 * math.pi * c / cams_per_pose
            el = rng.uniform(-0.15, 0.25)
            eye = (dist * math.sin(az) * math.cos(el), dist * math.sin(el) - 0.1, dist * math.cos(az) * math.cos(el))
            w, h = resolutions[v % len(resolutions)]
            cams.append(look_at_camera(w, h, eye))
            vp.append(p)
            v += 1
    return Batch(scene=scene, poses=np.stack(poses), lights=np.stack(lights), cameras=cams,
                 view_pose=np.asarray(vp, np.int32))


# Batched configurations: (scene config, poses, cameras per pose, resolutions, seed)
BATCH_CONFIGS = {
    # 32 poses x 4 cameras cycling 512x512, 1080x1080 and 1920 wide x 1080 high
    "c4_batch": dict(scene="c2_paper", n_poses=32, cams_per_pose=4,
                     resolutions=[(512, 512), (1080, 1080), (1920, 1080)], seed=2),
    # the same structure at test size, with image sizes that are no multiple of the tile edges
    "c4_small": dict(scene="c1_small", n_poses=3, cams_per_pose=2,
                     resolutions=[(64, 64), (100, 72), (136, 80)], seed=2),
}


def config_batch(name: str, **overrides) -> Batch:
    kw = dict(BATCH_CONFIGS[name])
    kw.update(overrides)
    scene = config_scene(kw.pop("scene"))
    return make_batch(scene, **kw)


# ---------------------------------------------------------------------------
# Displacement MLP weights (the trained weights are not available)
# ---------------------------------------------------------------------------
def mlp_weights(seed: int, pose_dims: int = 72, width: int = 256, n_freq: int = 64, freq_sd: float = 2.0) -> dict:
    """Seeded He-normal weights and small biases for the four layers, the
    output layer scaled to millimetre displacements, Gaussian frequencies
    (cycles per metre) for the Fourier features."""
    rng = np.random.default_rng(seed + 3000)

    def lin(o, i):
        return rng.normal(0.0, math.sqrt(2.0 / i), size=(o, i)), rng.normal(0.0, 0.01, size=o)

    W1, b1 = lin(width, 2 * n_freq + pose_dims)
    W2, b2 = lin(width, width)
    W3, b3 = lin(width, width)
    W4, b4 = lin(3, width)
    return dict(Bf=rng.normal(0.0, freq_sd, size=(n_freq, 3)), W1=W1, b1=b1, W2=W2, b2=b2, W3=W3, b3=b3,
                W4=W4 * 1e-3, b4=b4 * 1e-3)
