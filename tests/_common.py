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


def rel_err(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = max(float(np.abs(ref).max()), 1e-30)
    return float(np.abs(got - ref).max()) / scale


__all__ = ["O", "OP", "synth", "f32", "scene", "oracle_frame", "light_ordered_bits", "rel_err"]
