"""Host-side arithmetic of bench.py (no GPU): the workload counts that define
each stage's algorithmic work, the launch count it claims, the roofline
byte / op accounting and the rule that DRAM traffic from a committed ncu
capture is reported only while the kernel's source file is unchanged."""
import hashlib
import json
import os
import sys
import types

import numpy as np
import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _one_triangle_scene(R=4, F=1):
    """One direction looking down z (e1 = x, e2 = y), window [-1, 1]^2 at R^2:
    pixel centre i sits at s = (i + 1/2) 2/R - 1.  F copies of the triangle
    (-1,-1), (1,-1), (-1,1): front-facing, its box holds all R^2 centres, and
    it covers those with s + t <= 0."""
    xp = np.array([[-1.0, -1.0, 0.0], [1.0, -1.0, 0.0], [-1.0, 1.0, 0.0]])
    faces = np.tile(np.array([[0, 1, 2]], np.int32), (F, 1))
    av = types.SimpleNamespace(F=F, faces=faces, Nv=3)
    sc = types.SimpleNamespace(avatar=av, frames=np.array([[1.0, 0, 0, 0, 1.0, 0, 0, 0, 1.0]]), depth_res=R,
                               window_center=np.zeros(3), window_half=1.0)
    return xp, sc


def _frame(G=1000, NL=64, ntiles=4096, seed=0):
    g = torch.Generator().manual_seed(seed)
    r = types.SimpleNamespace()
    r.st = {"avatar": {"xg": torch.zeros(3, G)}, "light": {"w": torch.randn(NL, 3, generator=g)}}
    r.sh = {"cull": torch.randint(0, 2, (G,), dtype=torch.uint8, generator=g)}
    xp, sc = _one_triangle_scene(F=2000)
    r.sk = {"nd": torch.randn(3, G, generator=g), "xp": torch.as_tensor(xp.T.copy())}
    r.sb = types.SimpleNamespace(num_pairs=torch.tensor([5000], dtype=torch.int32),
                                 n_last=torch.randint(0, 5, (64, 64), dtype=torch.int32, generator=g),
                                 tile_range=torch.zeros(ntiles, 2, dtype=torch.int32))
    return r, sc


def test_visibility_work_counts_one_triangle_by_hand():
    """R = 4: the 16 centres are candidates, those with i + j <= 3 (10 of
    them, the diagonal on the edge included) are covered; 3 vertices are
    projected into the chunk cache and tested."""
    xp, sc = _one_triangle_scene()
    w = bench.visibility_work(xp, sc)
    assert w["counts"] == dict(setup=1, survivor=1, front=1, candidate=16, covered=10, cache_projection=3, test=3)
    ops = bench.VIS_OPS
    assert w["ops"] == (ops["setup"] + ops["survivor"] + ops["front"] + 16 * ops["candidate"] + 10 * ops["covered"]
                        + 3 * ops["cache_projection"] + 3 * ops["test"])
    # the reversed winding faces away: a survivor, but no candidates
    sc.avatar.faces = np.array([[0, 2, 1]], np.int32)
    w = bench.visibility_work(xp, sc)
    assert w["counts"]["front"] == 0 and w["counts"]["candidate"] == 0 and w["counts"]["survivor"] == 1


def test_workload_counts_follow_their_definitions():
    r, sc = _frame()
    st = bench.workload_stats(r, sc)
    cull = r.sh["cull"].numpy().astype(bool)
    cos = (r.st["light"]["w"].numpy() @ r.sk["nd"].numpy()) > 0
    assert st["front_gaussians"] == int((~cull).sum())
    assert st["lit_pairs_upper"] == int((cos & ~cull[None, :]).sum())
    assert st["pairs"] == 5000 and st["faces"] == 2000
    assert st["traversed_pairs"] == int(r.sb.n_last.sum())


@pytest.mark.parametrize("ntiles,passes", [(4096, 2), (255, 1), (256, 2), (70000, 3)])
def test_tile_sort_passes_and_launch_count(ntiles, passes):
    """The tile sort covers the tile ids and the no-tile key above them
    (2^bits > ntiles): 255 tiles fit one 8-bit pass, 256 take two."""
    r, sc = _frame(ntiles=ntiles)
    st = bench.workload_stats(r, sc)
    assert st["tile_sort_passes"] == passes
    # 23 kernels in every frame plus one onesweep pass per 8 bits of the tile id
    assert st["launches_per_frame"] == 23 + passes


def _scene(G=200_000, Nv=50_000, F=100_000, NL=512, D=512):
    av = types.SimpleNamespace(G=G, Nv=Nv, F=F)
    light = types.SimpleNamespace(A=np.zeros(NL))
    cam = types.SimpleNamespace(width=1024, height=1024)
    return types.SimpleNamespace(avatar=av, light=light, frames=np.zeros((D, 3, 3)), camera=cam)


def _stats(P=2_000_000):
    return {"front_gaussians": 100_000, "lit_pairs_upper": 20_000_000, "pairs": P, "faces": 100_000,
            "traversed_pairs": 30_000_000, "tile_sort_passes": 2, "launches_per_frame": 24,
            "visibility_work": {"ops": 4.5e9}}


ALU = {"fp32_tflops": 70.0, "int32_iadd3_tops": 20.0, "int32_lop3_tops": 20.0, "int32_imad_tops": 17.0,
       "sm_count": 152}


def test_roofline_accounting_and_dominant_stage(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))       # no committed traffic records
    sc, stats = _scene(), _stats()
    stages = {"skin": 0.040, "visibility": 0.500, "shade": 0.200, "bin": 0.180, "blend": 0.280}  # ms
    peaks = {"hbm_gbs": 6800.0, "sm_max_mhz": 2000.0}
    res = bench.roofline(stages, stats, sc, peaks, "measured", {}, ALU)
    out = res["stages"]
    # bytes / ops per unit as documented, divided by the stage time
    G, Nv, F, P = 200_000, 50_000, 100_000, 2_000_000
    assert out["skin"]["achieved"] == pytest.approx((140 * G + 164 * Nv) / 40e-6 / 1e9, rel=1e-3)
    assert out["bin"]["achieved"] == pytest.approx((G * (81 + 88 + 64 + 8) + P * (8 + 32 + 4)) / 180e-6 / 1e9,
                                                   rel=1e-3)
    assert out["visibility"]["achieved"] == pytest.approx(4.5e9 / 500e-6 / 1e12, rel=1e-3)
    assert out["blend"]["achieved"] == pytest.approx(15.0 * 30_000_000 / 280e-6 / 1e12, rel=1e-3)
    assert out["visibility"]["peak"] == pytest.approx(ALU["int32_iadd3_tops"], abs=0.1)
    assert out["shade"]["peak"] == pytest.approx(ALU["fp32_tflops"], abs=0.1)
    assert out["blend"]["peak"] == pytest.approx(ALU["fp32_tflops"], abs=0.1)
    for v in out.values():
        assert v["frac"] == pytest.approx(v["achieved"] / v["peak"], abs=2e-4)  # rounded to 4 places
        assert v["traffic"] is None
    assert res["stage"] == "visibility" and res["frac"] == out["visibility"]["frac"]


def test_traffic_is_reported_only_for_an_unchanged_source(tmp_path, monkeypatch):
    src = tmp_path / "kernel.cu"
    src.write_text("__global__ void k() {}\n")
    (tmp_path / "profiles").mkdir()
    rec = {"kernel": "k", "dram_bytes_per_launch": 1234.0, "source": "kernel.cu",
           "source_sha256": hashlib.sha256(src.read_bytes()).hexdigest()}
    (tmp_path / "profiles" / "ncu_traffic_c2.json").write_text(json.dumps({"kernels": {"blend": rec}}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    stages = {"skin": 0.040, "visibility": 0.500, "shade": 0.200, "bin": 0.180, "blend": 0.280}  # ms
    peaks = {"hbm_gbs": 6800.0}
    out = bench.roofline(stages, _stats(), _scene(), peaks, "measured", {}, ALU)["stages"]
    assert out["blend"]["traffic"] == 1234.0 and out["blend"]["traffic_kernel"] == "k"
    src.write_text("__global__ void k() { /* changed */ }\n")
    out = bench.roofline(stages, _stats(), _scene(), peaks, "measured", {}, ALU)["stages"]
    assert out["blend"]["traffic"] is None
