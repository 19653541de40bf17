"""Adjoint gradient dE2/dF and dE2/d(ia|jb): against the oracle's finite differences on a tiny
system, against central finite differences of the GPU energy (h = 1e-5) on 50 random elements
at No=16 Nv=160, the adjoint solve, and the autograd wrapper."""
import numpy as np
import pytest

import synth
from oracle import grad as ograd
from tests.gpu_util import handle_for

pytestmark = pytest.mark.gpu


def _pairs_F(N, rng, count):
    out = set()
    while len(out) < count:
        p, q = sorted(rng.integers(0, N, 2))
        out.add((int(p), int(q)))
    return sorted(out)


def _pairs_ov(No, Nv, rng, count):
    out = set()
    while len(out) < count:
        out.add((int(rng.integers(No)), int(rng.integers(Nv)), int(rng.integers(No)), int(rng.integers(Nv))))
    return sorted(out)


def _an_F(dF, p, q):
    return dF[p, q] + dF[q, p] if p != q else dF[p, p]


def _an_ov(dov, i, a, j, b):
    return dov[i, a, j, b] + dov[j, b, i, a] if (i, a) != (j, b) else dov[i, a, i, a]


def test_gradient_matches_oracle_finite_differences():
    No, Nv = 3, 6
    inst = synth.make_instance(No, Nv, 71, sigma_off=0.05)
    h = handle_for(inst)
    h.solve(tol=1e-13, maxit=2000)
    dF, dov, adj = h.grad(adjoint_solve=True)
    assert adj < 1e-9
    assert np.abs(dF - dF.T).max() < 1e-14
    N = No + Nv
    for p in range(N):
        for q in range(p, N):
            fd = ograd.fd_F(inst, p, q)
            an = _an_F(dF, p, q)
            assert abs(fd - an) <= 1e-6 * abs(fd) + 1e-8, (p, q, fd, an)
    rng = np.random.default_rng(3)
    for (i, a, j, b) in _pairs_ov(No, Nv, rng, 60):
        fd = ograd.fd_ovov(inst, i, a, j, b)
        an = _an_ov(dov, i, a, j, b)
        assert abs(fd - an) <= 1e-6 * abs(fd) + 1e-8, ((i, a, j, b), fd, an)


def _gpu_e2(inst):
    h = handle_for(inst)
    h.solve(tol=1e-13, maxit=3000)
    e = h.energy()["E2"]
    h.close()
    return e


def test_gradient_central_differences_c5():
    No, Nv, h_ = 16, 160, 1e-5
    inst = synth.make_instance(No, Nv, 5)
    hd = handle_for(inst)
    hd.solve(tol=1e-13, maxit=3000)
    dF, dov, adj = hd.grad(adjoint_solve=True)
    assert adj < 1e-8
    rng = np.random.default_rng(5)
    checked = 0
    for (p, q) in _pairs_F(No + Nv, rng, 25):
        vals = []
        for s in (1, -1):
            d = dict(inst)
            F = inst["F"].copy()
            F[p, q] += s * h_
            if p != q:
                F[q, p] += s * h_
            d["F"] = F
            vals.append(_gpu_e2(d))
        fd = (vals[0] - vals[1]) / (2 * h_)
        an = _an_F(dF, p, q)
        assert abs(fd - an) <= 1e-6 * abs(an) + 1e-7, (p, q, fd, an)
        checked += 1
    for (i, a, j, b) in _pairs_ov(No, Nv, rng, 25):
        vals = []
        for s in (1, -1):
            d = dict(inst)
            g = inst["ovov"].copy()
            g[i, a, j, b] += s * h_
            if (i, a) != (j, b):
                g[j, b, i, a] += s * h_
            d["ovov"] = g
            vals.append(_gpu_e2(d))
        fd = (vals[0] - vals[1]) / (2 * h_)
        an = _an_ov(dov, i, a, j, b)
        assert abs(fd - an) <= 1e-6 * abs(an) + 1e-7, ((i, a, j, b), fd, an)
        checked += 1
    assert checked == 50


def test_autograd_function():
    import torch
    from paper_2003_12923_gb300.autograd import esmp2_energy
    No, Nv = 4, 9
    inst = synth.make_instance(No, Nv, 72)
    t = {k: torch.from_numpy(inst[k]).cuda() for k in ("F", "ovov", "ooov", "ovvv", "C")}
    F = t["F"].clone().requires_grad_(True)
    ov = t["ovov"].clone().requires_grad_(True)
    e = esmp2_energy(F, ov, t["ooov"], t["ovvv"], t["C"], tol=1e-12)
    (2.0 * e).backward()
    h = handle_for(inst)
    h.solve(tol=1e-12)
    dF, dov, _ = h.grad()
    assert abs(float(e.detach()) - h.energy()["E2"]) < 1e-12
    assert np.abs(F.grad.cpu().numpy() - 2 * dF).max() < 1e-10 * max(1.0, np.abs(dF).max())
    assert np.abs(ov.grad.cpu().numpy() - 2 * dov).max() < 1e-10 * max(1.0, np.abs(dov).max())


def test_gradient_c5_against_stored_oracle_gradient():
    """No=16 Nv=160 (seed 5): float64 solve and esmp2_grad against the oracle's derivatives
    along sampled steps of F and (ia|jb), taken from the first-order equation at the oracle's
    own solution (tests/golden/o2_grad_c5.json), within 1e-6 relative."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "o2_grad_c5.json")
    if not os.path.exists(path):   # written offline by tests/golden/make_o2_reference.py
        pytest.skip("stored oracle gradient o2_grad_c5.json not generated")
    with open(path) as f:
        g = json.load(f)
    i = g["instance"]
    inst = synth.make_instance(i["No"], i["Nv"], i["seed"], sigma_off=i["sigma_off"])
    h = handle_for(inst)
    h.solve(tol=1e-12, maxit=3000)
    assert abs(h.energy()["E2"] - g["E2"]) < 1e-10
    dF, dov, _ = h.grad()
    for p, q, ref in g["dF_step"]:
        an = _an_F(dF, p, q)
        assert abs(an - ref) <= 1e-6 * abs(ref) + 1e-10, (p, q, an, ref)
    for ii, a, j, b, ref in g["dOVOV_step"]:
        an = _an_ov(dov, ii, a, j, b)
        assert abs(an - ref) <= 1e-6 * abs(ref) + 1e-10, ((ii, a, j, b), an, ref)
