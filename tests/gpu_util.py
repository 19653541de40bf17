"""Helpers shared by the GPU tests (seeded inputs and oracle references; no method arithmetic)."""
import numpy as np

import synth
from oracle import jw, o2, top


def handle_for(inst):
    from paper_2003_12923_gb300 import esmp2
    return esmp2.Handle(inst["F"], inst["ovov"], inst["ooov"], inst["ovvv"], inst["C"])


def masks(No, Nv):
    return np.stack([jw.block_mask(No, Nv, k) for k in jw.BLOCKS])


def random_block_vector(No, Nv, seed):
    """Random amplitudes with the storage symmetries of the layout (antisymmetric T, X, Y)
    and zeros on non-amplitude slots."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((5, No, No, Nv, Nv))
    for k in (0, 2, 3):
        a = x[k] - x[k].transpose(1, 0, 2, 3)
        x[k] = a - a.transpose(0, 1, 3, 2)
    return np.where(masks(No, Nv), x, 0.0)


def sample_indices(n, count, seed, shape=None, include=()):
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, n, count)
    return np.unique(np.concatenate([idx, np.asarray(include, dtype=np.int64)]))
