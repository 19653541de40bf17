"""The benchmark workload's size (No=30, Nv=400; 720M amplitudes): sigma elements sampled at
random, plus the corners of every block, against the oracle evaluated element by element,
for the float64, float64-exact tensor-core and bf16 forms.  The sigma operator does not
involve the two-electron integrals, so the handle is created with zero integral blocks."""
import numpy as np
import pytest

import synth
from oracle import o2, top
from tests.gpu_util import random_block_vector, sample_indices

pytestmark = pytest.mark.gpu


def test_sigma_sampled_at_benchmark_size():
    import torch
    from paper_2003_12923_gb300 import esmp2
    No, Nv, seed = 30, 400, 3
    F = synth.fock(No, Nv, seed, 1e-3)
    C = synth.singles_coefficients(F, No, Nv, seed)

    def zeros(*shape):
        return torch.zeros(shape, dtype=torch.float64, device="cuda")

    h = esmp2.Handle(torch.from_numpy(F).cuda(), zeros(No, Nv, No, Nv), zeros(No, No, No, Nv),
                     zeros(No, Nv, Nv, Nv), torch.from_numpy(C).cuda())
    x = random_block_vector(No, Nv, 77).reshape(-1)
    B = No * No * Nv * Nv
    corners = [k * B + off for k in range(5)
               for off in (0, Nv - 1, (Nv - 1) * Nv, B - 1, (No * No - 1) * Nv * Nv + 1)]
    idx = sample_indices(x.size, 4000, 5, include=corners)
    U, lam, Wv = top.top_basis(top.normalise_singles(C))
    prep = {"No": No, "Nv": Nv, "F": top.transform_fock(F, U, Wv), "lam": lam,
            "ovov": np.zeros((No, Nv, No, Nv)), "ooov": np.zeros((No, No, No, Nv)),
            "ovvt": np.zeros((No, Nv, Nv, No))}
    ref = o2.O2(prep).sigma_at(x, idx)
    scale = float(np.abs(ref).max())
    xt = torch.from_numpy(x).cuda()
    del x
    it = torch.from_numpy(idx).cuda()
    # float64 and float64-exact forms to float64 accuracy; the bf16 form within its rounding
    for prec, rel in ((esmp2.FP64, 1e-11), (esmp2.FP64_TC, 1e-11), (esmp2.MIXED_BF16, 2e-2)):
        y = h.sigma(xt, prec).reshape(-1)[it].cpu().numpy()
        err = float(np.abs(y - ref).max())
        assert err <= rel * scale, (prec, err, scale)
    h.close()
