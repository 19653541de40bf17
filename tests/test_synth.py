"""The seeded input generator against its published definition and the workload recipe."""
import numpy as np

import synth


def _mix64(z):
    M = (1 << 64) - 1
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
    return z ^ (z >> 31)


def test_splitmix64_reference_value():
    # SplitMix64 seeded with 0: the first output is 0xE220A8397B1DCDAF (Steele et al. 2014).
    assert _mix64(0x9E3779B97F4A7C15) == 0xE220A8397B1DCDAF


def _normal_py(seed, stream, n):
    import math
    G = 0x9E3779B97F4A7C15
    M = (1 << 64) - 1
    key = _mix64((seed * G + _mix64(stream + 1)) & M)
    d = lambda k: _mix64((key + (k + 1) * G) & M)
    u1 = ((d(2 * n) >> 11) + 1.0) * 2.0 ** -53
    u2 = (d(2 * n + 1) >> 11) * 2.0 ** -53
    return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


def test_c_generator_matches_definition():
    for (seed, stream, n) in [(0, 2, 0), (5, 2, 123456), (1, 1, 77), (9, 3, 4)]:
        assert abs(synth._load().synth_normal(seed, stream, n) - _normal_py(seed, stream, n)) < 1e-15


def test_eri_symmetry_and_blocks():
    No, Nv = 3, 5
    e = synth.eri_block("full", No, Nv, seed=4)
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (3, 2, 1, 0)]:
        assert np.array_equal(e, e.transpose(perm))
    assert np.array_equal(synth.eri_block("ovov", No, Nv, 4), e[:No, No:, :No, No:])
    assert np.array_equal(synth.eri_block("ooov", No, Nv, 4), e[:No, :No, :No, No:])
    assert np.array_equal(synth.eri_block("ovvv", No, Nv, 4), e[:No, No:, No:, No:])
    assert synth.eri_scalar(4, 1e-2, 1, 5, 2, 7) == e[1, 5, 2, 7]


def test_instance_recipe():
    inst = synth.make_instance(6, 30, seed=0)
    F, C = inst["F"], inst["C"]
    assert np.array_equal(F, F.T)
    d = np.diag(F)
    assert d[:6].min() >= -2.0 and d[:6].max() <= -0.3
    assert d[6:].min() >= 0.2 and d[6:].max() <= 3.0
    lam = np.linalg.svd(C, compute_uv=False)
    assert abs(2 * np.sum(C ** 2) - 1) < 1e-12
    assert abs(lam[0] ** 2 / np.sum(lam ** 2) - 0.9) < 1e-9
    inst2 = synth.make_instance(6, 30, seed=0)
    assert np.array_equal(inst2["ovvv"], inst["ovvv"]) and np.array_equal(inst2["C"], C)


def test_batch_shapes():
    sh = synth.batch_shapes(64)
    assert len(sh) == 64
    for No, Nv, s in sh:
        assert 8 <= No <= 32 and 8 * No - 1 <= Nv <= 14 * No + 1
