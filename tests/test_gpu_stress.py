"""The stress configuration (200k-vertex mesh, 1M Gaussians, 32 x 64 light,
1,024 visibility directions at 512^2, 2048 x 2048 image): the tensor-core
shading (BF16 D and S, FP32 accumulation) against the FP32 CUDA-core shading
of the same frame at max-abs pixel error <= 1e-3, with FP32 and with BF16
attribute storage, and the training step (forward on the tensor cores,
FP32 adjoints) against the FP32 training step.  At 2048^2 a Gaussian of the
configuration's size spans about fifty 16-pixel tiles, so the pair buffers
hold 96 pairs per Gaussian."""
import numpy as np
import pytest

from _common import scene

CAP = 96 * 1_000_000

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    from paper_2407_10707_gb300 import render
    return render


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_stress_tensor_core_frame_matches_fp32(gpu, dtype):
    render = gpu
    sc = scene("c5_stress")
    st = render.scene_tensors(sc, "cuda", attr_dtype=dtype)
    r32 = render.Renderer(st, pair_capacity=CAP)
    img32 = r32.forward().clone()
    r32.check()
    rtc = render.Renderer(st, shade_tc=True, pair_capacity=CAP)
    imgtc = rtc.forward().clone()
    rtc.check()
    torch.cuda.synchronize()
    assert int(r32.sb.num_pairs.item()) > 1_000_000
    err = float((imgtc - img32).abs().max())
    assert err <= 1e-3, err
    assert float(img32.max()) > 0.1  # the frame is not empty


def test_stress_train_step_tensor_core_vs_fp32(gpu):
    render = gpu
    sc = scene("c5_stress")
    st = render.scene_tensors(sc, "cuda")
    target = (render.Renderer(st, pair_capacity=CAP).forward().detach().clone() * 0.9).contiguous()
    ts32 = render.TrainStep(st, target, pair_capacity=CAP)
    g32 = {k: v.clone() for k, v in ts32.grads().items()}
    l32 = float(ts32.loss.item())
    ts32.check()
    del ts32
    tstc = render.TrainStep(st, target, shade_tc=True, pair_capacity=CAP)
    gtc = {k: v.clone() for k, v in tstc.grads().items()}
    ltc = float(tstc.loss.item())
    tstc.check()
    torch.cuda.synchronize()
    assert abs(ltc - l32) <= 1e-3 * abs(l32)
    for k in g32:
        a, b = g32[k].float(), gtc[k].float()
        scale = float(a.abs().max())
        assert scale > 0, k
        assert float((a - b).abs().max()) <= 1e-2 * scale, k
