"""mm_apply_A_noalloc: A x without any allocation by the library.

Some callers cannot let the library allocate device memory (fixed pools or arenas, real-time
loops, hosts that account for every byte themselves).  mm_apply_A_noalloc takes its working space
from a fixed array compiled into libmm instead of plan buffers grown with cudaMalloc.  This file
checks, through the C ABI, that it returns what mm_apply_A returns (within the tolerances of the
other parity tests) on two calls in a row (the second call must not see the first call's
leftovers), and that a working set beyond the fixed array is refused with a clear error.
It is collected last so that a failure here cannot hide the results of the other GPU tests.
"""
import numpy as np
import pytest
import torch

import synth
from gpu_helpers import cuda, mm, plans, rel_max

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,tol", [(0, 1e-11), (1, 2e-5), (3, 2e-5)])
@pytest.mark.parametrize("nrhs", [1, 3])
def test_noalloc_matches_apply_A_twice(precision, tol, nrhs):
    prob = synth.random_problem(4, [70001, 5, 33000, 40000], 300, 1024, seed=21, gap_frac=0.02,
                                hits_per_pix_min=4)
    gp, op, _ = plans(prob, precision=precision)
    m = mm()
    rng = np.random.default_rng(nrhs + 10 * precision)
    for call in range(2):
        x = cuda(rng.standard_normal((nrhs, op.n_obs, 3)))
        y_ref = torch.empty_like(x)
        y = torch.full_like(x, float("nan"))
        m.mm_apply_A(gp, x, y_ref)
        m.mm_apply_A_noalloc(gp, x, y)
        torch.cuda.synchronize()
        assert torch.isfinite(y).all()
        assert rel_max(y.cpu().numpy(), y_ref.cpu().numpy()) < tol, f"call {call}"


def test_noalloc_rejects_oversized_working_set():
    m = mm()
    prob = synth.random_problem(2, [20000, 20000], 300, 64, seed=22, hits_per_pix_min=4)
    gp, op, _ = plans(prob)
    nrhs = 524288 // op.n_obs + 1            # FP64: nrhs * n_obs > 524,288
    x = torch.zeros(nrhs, op.n_obs, 3, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(m.MMError) as e:
        m.mm_apply_A_noalloc(gp, x, y)
    assert e.value.code == m.MM_EINVAL and "working space" in str(e.value)


def test_noalloc_refuses_df64_plans():
    """An MM_DF64 plan's operator is double-float arithmetic over an N-sample buffer, which the
    fixed array cannot hold: the call is refused rather than run in other arithmetic."""
    m = mm()
    prob = synth.random_problem(2, [20000, 20000], 300, 64, seed=23, hits_per_pix_min=4)
    gp, op, _ = plans(prob, precision=m.MM_DF64)
    x = torch.zeros(1, op.n_obs, 3, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(m.MMError) as e:
        m.mm_apply_A_noalloc(gp, x, y)
    assert e.value.code == m.MM_EINVAL and "MM_DF64" in str(e.value)
