"""Whole-frame composition of the FP64 C oracle stages (test infrastructure).

frame(scene) runs, in the paper's order (Sec. 3.1-3.2): forward kinematics,
skinning (Eq. 1 + LBS), depth-map visibility of the posed mesh, shading
(Eq. 2 + App. A), EWA projection and brute-force compositing.  The scene is
any object with the attributes produced by the seeded input generator
(avatar, light, frames, dmap, camera, depth_res, window_center, window_half,
vis_bias); nothing here is imported by the product path.
"""
from __future__ import annotations

import numpy as np

from . import oracle as O


def f32(a):
    """Round to FP32 and back: the values an FP32 stage input actually holds."""
    return np.asarray(a, np.float32).astype(np.float64)


def frame(scene, pixels=None, bits=None):
    av = scene.avatar
    bone = O.fk(av.parents, av.joints, av.pose)
    sk = O.skin(av, bone)
    if bits is None:
        bits = O.visibility(f32(sk["xp"]), av.faces, f32(scene.frames.reshape(-1, 9)),
                            scene.window_center, scene.window_half, scene.vis_bias,
                            scene.depth_res)
    n_dirs = scene.frames.shape[0]
    color, radiance, cull = O.shade(sk["xd"], sk["nd"], sk["ag"], sk["rg"], sk["pg"], sk["ubar"],
                                    av.knn, bits, scene.light.L, scene.light.A, scene.light.w,
                                    scene.dmap, scene.camera.center, n_dirs)
    pr = O.project(sk["xd"], sk["cov"], av.opacity, cull, scene.camera)
    cam = scene.camera
    rgb, T, count, amb = O.composite(pr["mean2d"], pr["conic"], av.opacity, color, pr["depth"],
                                     pr["valid"], cam.width, cam.height, pixels)
    return dict(bone=bone, skin=sk, bits=bits, color=color, radiance=radiance, cull=cull,
                proj=pr, rgb=rgb, T=T, count=count, amb=amb)
