"""Helpers shared by the GPU tests (seeded inputs and oracle references; no method arithmetic)."""
import numpy as np

import synth
from oracle import jw, o2, top


def handle_for(inst):
    from paper_2003_12923_gb300 import esmp2
    return esmp2.Handle(inst["F"], inst["ovov"], inst["ooov"], inst["ovvv"], inst["C"])


def masks(No, Nv):
    return np.stack([jw.block_mask(No, Nv, k) for k in jw.BLOCKS])


def random_block_vector(No, Nv, seed, singlet=True):
    """Random amplitudes with the storage symmetries of the layout (antisymmetric T, X, Y)
    and zeros on non-amplitude slots; singlet=True also gives S the spin-flip symmetry
    S_ij^ab = S_ji^ba that every vector of the singlet problem has."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((5, No, No, Nv, Nv))
    for k in (0, 2, 3):
        a = x[k] - x[k].transpose(1, 0, 2, 3)
        x[k] = a - a.transpose(0, 1, 3, 2)
    if singlet:
        x[1] = 0.5 * (x[1] + x[1].transpose(1, 0, 3, 2))
    return np.where(masks(No, Nv), x, 0.0)


def sample_indices(n, count, seed, shape=None, include=()):
    rng = np.random.default_rng(seed)
    idx = rng.integers(0, n, count)
    return np.unique(np.concatenate([idx, np.asarray(include, dtype=np.int64)]))


def indefinite_instance(No, Nv, seed, shift=7.0):
    """A synthetic instance whose first-order operator is indefinite: every occupied orbital
    energy is raised by `shift` above the virtual ones (an intruder-state setting), so most
    doubles and L-triples have negative zeroth-order excitation energies.  Input shaping only."""
    inst = synth.make_instance(No, Nv, seed)
    F = inst["F"].copy()
    F[np.arange(No), np.arange(No)] += shift
    inst["F"] = F
    inst["C"] = synth.singles_coefficients(F, No, Nv, seed)
    return inst
