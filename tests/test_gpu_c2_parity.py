"""Parity at the paper-scale frame, in the configuration the benchmark times.

The frame: 50k-vertex body mesh, 200k Gaussians stored in the order of their
nearest vertex (render.spatially_ordered), 16 x 32 environment light stored
in 4 x 8 patches (render.light_ordered), the faces by normal within each
raster chunk (render.faces_ordered), 512
visibility directions at 256^2 (one-sided raster of the closed body), one
1024 x 1024 camera, 16-pixel tiles; the overlapped frame (cull, projection and
binning on a second stream) replayed from its CUDA graph.  The oracle runs on
the same reordered avatar, light and faces (the Gaussian order checked
equal to numpy's stable sort).

Every stage is compared with the FP64 oracle on the GPU's own inputs (the
stage chain of tests/_chain.py): the visibility bits of all 512 directions
and every tile-list entry bit for bit, the colours of all 200k Gaussians and
4,096 sampled pixels within 2e-4 (pixels the oracle flags ambiguous are
excluded and counted, no other exemption).  Against the pure oracle chain
(FP64 from the avatar on) every difference above 2e-4 must be explained by a
visibility bit or cull flag that FP32 skinning moved across an integer step.
"""
import numpy as np
import pytest

from _chain import chain_check, end_to_end_report
from _common import OP, scene

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def frame():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    from paper_2407_10707_gb300 import render
    from _common import synth
    sc0 = scene("c2_paper")
    st, order = render.spatially_ordered(render.scene_tensors(sc0))   # the benchmark's storage orders
    np_order = synth.nearest_vertex_order(sc0)
    assert np.array_equal(order.cpu().numpy(), np_order)
    lorder = synth.latlong_patch_order(sc0.light.rows, sc0.light.cols)
    st, _ = render.light_ordered(st, lorder)
    forder = synth.face_normal_order(sc0.avatar.xv, sc0.avatar.faces)
    st, _ = render.faces_ordered(st, forder)
    sc = synth.permute_faces(synth.permute_lights(synth.permute_gaussians(sc0, np_order), lorder), forder)
    r = render.Renderer(st, tile=16)              # the benchmark's renderer and tile edge
    r.capture()
    for _ in range(3):
        r.replay()
    torch.cuda.synchronize()
    r.check()
    # 4,096 pixels: 3,072 among those the body covers (final transmittance < 1),
    # 1,024 anywhere in the image
    T = r.sb.T_final.reshape(-1).cpu().numpy()
    rng = np.random.default_rng(21)
    covered = np.flatnonzero(T < 1.0)
    first = rng.choice(covered, 3072, replace=False)
    rest = np.setdiff1d(np.arange(T.size), first)
    pix = np.sort(np.concatenate([first, rng.choice(rest, 1024, replace=False)])).astype(np.int32)
    return sc, r, pix


def test_c2_frame_every_stage_on_the_gpus_own_inputs(frame):
    sc, r, pix = frame
    rep = chain_check(r, sc, pixels=pix)
    rep.pop("gpu")
    print("c2 stage chain:", rep)
    assert rep["visibility_directions"] == 512
    assert rep["shaded_gaussians"] > 50_000
    assert rep["pixels_covered"] > 2_500


def test_c2_frame_against_the_pure_oracle_chain(frame):
    sc, r, pix = frame
    from _chain import gpu_buffers
    ref = OP.frame(sc, pixels=pix)
    rep = end_to_end_report(gpu_buffers(r), sc, ref, pixels=pix)
    print("c2 end to end:", rep)
