"""Shared helpers of the test suite: scene construction and oracle runs.

Inputs come from the seeded generator (paper_2407_10707_gb300.synth); the
expected values come from the FP64 oracle only.
"""
import functools

import numpy as np

from oracle import oracle as O
from oracle import pipeline as OP
from paper_2407_10707_gb300 import synth


def f32(a):
    return np.asarray(a, np.float32)


@functools.lru_cache(maxsize=8)
def scene(name, **kw):
    return synth.config_scene(name, **dict(kw))


@functools.lru_cache(maxsize=8)
def oracle_frame(name):
    return OP.frame(scene(name))


def light_ordered_bits(bits_view, dmap):
    """Re-order viewpoint-ordered oracle bits [Nv, D/32] per light k via d(k)."""
    Nv = bits_view.shape[0]
    NL = len(dmap)
    b = np.unpackbits(bits_view.view(np.uint8), bitorder="little").reshape(Nv, -1)
    out = np.zeros((Nv, ((NL + 31) // 32) * 32), np.uint8)
    out[:, :NL] = b[:, dmap]
    return np.packbits(out, bitorder="little").view(np.uint32).reshape(Nv, -1)


def bf16_round(a):
    """FP32 -> bfloat16 (round to nearest, ties to even) -> FP32, by bit
    arithmetic on finite values: the value a BF16-stored attribute holds."""
    x = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    r = ((x + 0x7FFF + ((x >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).reshape(np.shape(a))


BF16_ATTRS = ("logscale", "quat", "opacity", "av", "rv", "pv")


def bf16_scene(sc):
    """The scene whose learnable attributes hold their BF16-rounded values."""
    import dataclasses
    av = dataclasses.replace(sc.avatar, **{k: bf16_round(getattr(sc.avatar, k)) for k in BF16_ATTRS})
    return dataclasses.replace(sc, avatar=av)


def rel_err(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = max(float(np.abs(ref).max()), 1e-30)
    return float(np.abs(got - ref).max()) / scale


__all__ = ["O", "OP", "synth", "f32", "scene", "oracle_frame", "light_ordered_bits", "rel_err", "bf16_round",
           "bf16_scene", "BF16_ATTRS"]


LOG2_ALPHA_MIN = float(np.log2(1.0 / 255.0))


def check_tile_lists(pairs, tile_range, start, lst, mean2d, conic, opacity, W, H, tile, pixels=None,
                     margin=1e-4):
    """The GPU's tile lists against the oracle's rect lists (orc_bin).

    Binning emits a pair for every tile of a Gaussian's rect (so the pair
    count is the oracle's) but lists only the tiles its ellipse can reach;
    which of the others it drops is free, as they add nothing to any pixel.
    Checked here: (1) each GPU tile list is the oracle's list of that tile
    with some entries dropped, in the oracle's (depth, index) order; (2) at
    every pixel centre checked (pixels, flat indices; default all) every
    Gaussian of the oracle's tile list whose log2 alpha, in FP64 from the
    FP32 projection, reaches log2(1/255) + margin is in the GPU's list.
    Returns (kept pairs, oracle pairs, pairs required at the pixels)."""
    ntiles = len(start) - 1
    G = max(int(lst.max()) + 1 if len(lst) else 1, int(pairs.max()) + 1 if len(pairs) else 1)
    otile = np.repeat(np.arange(ntiles), np.diff(start))
    okey = otile.astype(np.int64) * G + lst
    order = np.argsort(okey, kind="stable")
    cnt = tile_range[:, 1] - tile_range[:, 0]
    assert np.all(cnt >= 0) and np.all(cnt <= np.diff(start)), "a tile list is longer than the oracle's"
    ne = cnt > 0
    gtile = np.repeat(np.arange(ntiles)[ne], cnt[ne])
    gidx = np.concatenate([np.arange(a, b) for a, b in tile_range[ne]]) if ne.any() else np.zeros(0, np.int64)
    gg = pairs[gidx]
    gkey = gtile.astype(np.int64) * G + gg
    at = np.searchsorted(okey[order], gkey)
    found = (at < len(okey)) & (okey[order][np.minimum(at, len(okey) - 1)] == gkey)
    assert found.all(), f"{int((~found).sum())} listed pairs are not in the oracle's lists"
    pos = order[at]                                     # place of each listed pair in the oracle's list
    same = gtile[1:] == gtile[:-1]
    assert np.all(np.diff(pos)[same] > 0), "a tile list is out of the oracle's (depth, index) order"
    # completeness at the pixel centres
    pix = np.arange(W * H) if pixels is None else np.asarray(pixels)
    px, py = pix % W, pix // W
    ntx = (W + tile - 1) // tile
    tpix = (py // tile) * ntx + px // tile
    need = 0
    L2E = 1.0 / np.log(2.0)
    mean2d = np.asarray(mean2d, np.float64)
    conic = np.asarray(conic, np.float64)
    lo2 = np.log2(np.asarray(opacity, np.float64))
    kept = set(gkey.tolist())
    for c0 in range(0, len(pix), 512):
        tp, xs, ys = tpix[c0:c0 + 512], px[c0:c0 + 512] + 0.5, py[c0:c0 + 512] + 0.5
        n = start[tp + 1] - start[tp]
        rep = np.repeat(np.arange(len(tp)), n)
        ent = np.concatenate([lst[start[t]:start[t + 1]] for t in tp]) if n.sum() else np.zeros(0, np.int64)
        dx = xs[rep] - mean2d[ent, 0]
        dy = ys[rep] - mean2d[ent, 1]
        l2a = (-0.5 * L2E * conic[ent, 0] * dx * dx - L2E * conic[ent, 1] * dx * dy
               - 0.5 * L2E * conic[ent, 2] * dy * dy + lo2[ent])
        req = l2a >= LOG2_ALPHA_MIN + margin
        rk = tp[rep[req]].astype(np.int64) * G + ent[req]
        need += int(req.sum())
        miss = [k for k in np.unique(rk).tolist() if k not in kept]
        assert not miss, f"{len(miss)} pairs that reach a pixel are not listed, e.g. tile {miss[0] // G}, " \
                         f"Gaussian {miss[0] % G}"
    return len(gkey), len(lst), need
