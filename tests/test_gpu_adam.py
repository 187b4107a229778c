"""The Adam update (avatar_adam) against the FP64 oracle.

Tolerances: the kernel forms the moments and the step in FP32 with fused
multiply-adds; each is a handful of roundings (relative 2^-24 each), so m
is checked to 2^-21 of the magnitude of its two summands (which may
cancel), v (a sum of non-negative terms) to 2^-20 relative, and the
parameter to 2^-22 of its magnitude plus 1e-5 of the learning rate; each
step is checked from the kernel's own state after the previous one.  A bfloat16 parameter
equals the oracle's rounded value, or lies one bfloat16 step from it when
the exact update falls within FP32 error of a rounding boundary (at most
0.1 % of the elements)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

f32 = lambda x: float(np.float32(x))  # the kernel's FP32 hyper-parameters
HP = dict(b1=f32(0.9), b2=f32(0.999), eps=f32(1e-15))


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build()
    from paper_2407_10707_gb300 import api
    return api


def test_adam_matches_oracle(gpu):
    api = gpu
    from oracle import adam as AD
    from oracle import mlp as M
    rng = np.random.default_rng(21)
    sizes = [1, 7, 1000, 4099, 262147]
    lrs = [1e-2, 1e-3, 5e-2, 1.6e-4, 2.5e-3]
    dtypes = [torch.float32, torch.float32, torch.bfloat16, torch.float32, torch.float32]
    p0 = [rng.normal(size=n).astype(np.float32) for n in sizes]
    P = [torch.as_tensor(x, device="cuda").to(dt) for x, dt in zip(p0, dtypes)]
    Mm = [torch.zeros(n, device="cuda") for n in sizes]
    V = [torch.zeros(n, device="cuda") for n in sizes]
    ref = [(M.bf16(x) if dt == torch.bfloat16 else x.astype(np.float64), np.zeros(len(x)), np.zeros(len(x)))
           for x, dt in zip(p0, dtypes)]
    for t in range(1, 4):
        g = [(rng.normal(size=n) * 10.0 ** rng.uniform(-4, 1, size=n)).astype(np.float32) for n in sizes]
        G = [torch.as_tensor(x, device="cuda") for x in g]
        api.avatar_adam([(P[k], G[k], Mm[k], V[k], lrs[k]) for k in range(len(sizes))], t)
        torch.cuda.synchronize()
        for k in range(len(sizes)):
            bf = dtypes[k] == torch.bfloat16
            pr, mr, vr = AD.step(ref[k][0], g[k].astype(np.float64), ref[k][1], ref[k][2], t, f32(lrs[k]), bf16=bf,
                                 **HP)
            got_p = P[k].float().cpu().numpy().astype(np.float64)
            # m: a couple of roundings relative to its two summands (they may cancel)
            scale_m = HP["b1"] * np.abs(ref[k][1]) + (1 - HP["b1"]) * np.abs(g[k])
            assert np.all(np.abs(Mm[k].cpu().numpy() - mr) <= 2.0 ** -21 * scale_m)
            np.testing.assert_allclose(V[k].cpu().numpy(), vr, rtol=2.0 ** -20, atol=1e-30)
            if bf:
                diff = got_p != pr
                assert diff.mean() <= 1e-3
                step = np.abs(pr) * 2.0 ** -7  # at most one bfloat16 step apart
                assert np.all(np.abs(got_p - pr)[diff] <= step[diff] + 1e-30)
            else:
                assert np.all(np.abs(got_p - pr) <= 2.0 ** -22 * np.abs(pr) + 1e-5 * lrs[k])
            # the next step starts from the kernel's own state, so each check covers one step's roundings
            ref[k] = (got_p, Mm[k].cpu().numpy().astype(np.float64), V[k].cpu().numpy().astype(np.float64))


def test_adam_unaligned_tensors_take_the_scalar_path(gpu):
    api = gpu
    from oracle import adam as AD
    rng = np.random.default_rng(3)
    base = torch.as_tensor(rng.normal(size=1001).astype(np.float32), device="cuda")
    p = base[1:]                      # 4 bytes past an aligned start
    g = torch.as_tensor(rng.normal(size=1000).astype(np.float32), device="cuda")
    m, v = torch.zeros(1001, device="cuda")[1:], torch.zeros(1001, device="cuda")[1:]
    first = float(base[0])
    pr, _, _ = AD.step(p.cpu().numpy(), g.cpu().numpy(), np.zeros(1000), np.zeros(1000), 1, f32(0.01), **HP)
    api.avatar_adam([(p, g, m, v, 0.01)], 1)
    torch.cuda.synchronize()
    assert np.all(np.abs(p.cpu().numpy() - pr) <= 2.0 ** -22 * np.abs(pr) + 1e-7)
    assert float(base[0]) == first  # the element before the slice is untouched


def test_train_step_update_applies_adam_to_every_group(gpu):
    """TrainStep.update() moves every trainable tensor by the oracle's Adam
    step of the gradients the step left."""
    from oracle import adam as AD
    from paper_2407_10707_gb300 import render
    from _common import scene
    sc = scene("c3_fd")
    st = render.scene_tensors(sc, "cuda")
    r = render.Renderer(st)
    target = (r.forward().detach().clone() * 0.8).contiguous()
    ts = render.TrainStep(st, target, adam=True)
    ts.step()
    torch.cuda.synchronize()
    before = {k: p.detach().float().cpu().numpy().astype(np.float64) for k, p in ts.opt.params.items()}
    grads = {k: g.detach().cpu().numpy().astype(np.float64) for k, g in ts.grads().items()}
    ts.update()
    torch.cuda.synchronize()
    for k, p in ts.opt.params.items():
        want, _, _ = AD.step(before[k], grads[k], 0.0, 0.0, 1, f32(render.ADAM_LR[k]), **HP)
        got = p.detach().float().cpu().numpy()
        assert np.all(np.abs(got - want) <= 2.0 ** -22 * np.abs(want) + 1e-5 * render.ADAM_LR[k]), k


def test_adam_edge_cases(gpu):
    api = gpu
    from paper_2407_10707_gb300 import _lib as L
    api.avatar_adam([], 1)  # no groups: nothing to do
    e = torch.zeros(0, device="cuda")
    api.avatar_adam([(e, e, e, e, 0.1)], 1)  # an empty group
    # sixteen groups (the limit) in one launch, each a one-element tensor
    ps = [torch.full((1,), float(k), device="cuda") for k in range(16)]
    gs = [torch.ones(1, device="cuda") for _ in range(16)]
    ms = [torch.zeros(1, device="cuda") for _ in range(16)]
    vs = [torch.zeros(1, device="cuda") for _ in range(16)]
    api.avatar_adam([(ps[k], gs[k], ms[k], vs[k], 0.5) for k in range(16)], 1)
    torch.cuda.synchronize()
    assert all(abs(float(ps[k]) - (k - 0.5)) < 1e-6 for k in range(16))  # first step: lr sign(g)
    with pytest.raises(ValueError):
        api.avatar_adam([(ps[0], gs[0], ms[0], vs[0], 0.5)] * 17, 1)
    with pytest.raises(L.AvatarError):
        api.avatar_adam([(ps[0], gs[0], ms[0], vs[0], 0.5)], 0)  # steps count from 1
