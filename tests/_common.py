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
