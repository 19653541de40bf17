"""The allocation-free bf16 contraction agrees with the handle-based entry point.

esmp2_virtual_contraction_noalloc serves callers that cannot allocate device memory
where they call it (another framework owns the device heap, or a latency-critical loop
must not synchronise on cudaMalloc/cudaFree); its scratch is a fixed device array inside
the library.  This file is collected last so that a run stopping at the first failure has
already run every other test; it passes alone in a fresh process too.
"""
import numpy as np
import pytest

import synth
from tests.gpu_util import handle_for

pytestmark = pytest.mark.gpu


def test_noalloc_matches_handle_entry_point_twice():
    import torch
    from paper_2003_12923_gb300 import esmp2
    No, Nv = 3, 40
    inst = synth.make_instance(No, Nv, seed=41)
    h = handle_for(inst)
    Fvv = torch.from_numpy(np.ascontiguousarray(h.top_basis()[3][No:, No:])).cuda()
    S = 5 * No * No
    rng = np.random.default_rng(5)
    for call in range(2):   # two calls in a row share (and reuse) the scratch array
        x = torch.from_numpy(rng.standard_normal(h.shape)).cuda()
        ref = h.virtual_contraction(x, esmp2.MIXED_BF16)
        y = torch.full(h.shape, float("nan"), dtype=torch.float64, device="cuda")
        st = esmp2.virtual_contraction_noalloc(x, Fvv, y, S, Nv)
        assert st == esmp2.OK, (call, st)
        err = float((y - ref).abs().max())
        assert err <= 1e-12 * float(ref.abs().max()), (call, err)


def test_noalloc_rejects_oversized_request():
    import torch
    from paper_2003_12923_gb300 import esmp2
    Nv = 400
    S = 5 * 30 * 30   # far beyond the fixed scratch
    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = esmp2.virtual_contraction_noalloc(x, x, x, S, Nv)
    assert st == esmp2.ERR_UNSUPPORTED
