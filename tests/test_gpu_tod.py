"""mm_solve_tod: the map from the TOD in one call.  On an MM_FP32_DF64 plan with FP32 iterations
the right-hand side comes from the FP32 operators and every true residual from the data,
P^T N^-1 G (d - P x), in double-float; the map must still match the FP64 oracle's PCG at the same
tol within the mixed-precision tolerance, with a true residual below tol.  Other plan precisions run
the FP64-class right-hand side and PCG, and must match the oracle within the FP64 tolerance."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from gpu_helpers import mm, plans

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny():
    cfg = synth.tiny_config()
    prob = synth.make_ground_problem(cfg)
    nb = synth.to_numpy(prob)
    op = O.make_plan(nb["pix"], nb["psi"], nb["block_len"], nb["band"], nb["n_pix"])
    ref = O.pcg(op, O.rhs(op, nb["d"]), tol=cfg.tol, max_iter=5000)
    return cfg, prob, nb, op, ref


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("fp32_d", [False, True])
def test_tod_solve_mixed_matches_oracle(tiny, fp32_d):
    cfg, prob, nb, op, ref = tiny
    m = mm()
    gp, _, _ = plans(prob, precision=m.MM_FP32_DF64)
    d = torch.as_tensor(nb["d"].astype(np.float32) if fp32_d else nb["d"], device="cuda")
    x = torch.empty(op.n_obs, 3, dtype=torch.float64, device="cuda")
    info = m.mm_solve_tod(gp, d, x, tol=cfg.tol, max_iter=5000, precision=m.MM_FP32)[0]
    assert info.status == 0 and info.true_rel_res < cfg.tol
    assert info.n_apply64 >= 1   # the double-float residual certified the stop
    r = ref if not fp32_d else O.pcg(op, O.rhs(op, nb["d"].astype(np.float32).astype(np.float64)),
                                     tol=cfg.tol, max_iter=5000)
    assert rel(x.cpu().numpy(), r.x) < 1e-5


def test_tod_solve_equals_rhs_then_pcg(tiny):
    """Same map as mm_rhs + mm_pcg_solve on the same plan (both certified to tol)."""
    cfg, prob, nb, op, ref = tiny
    m = mm()
    gp, _, _ = plans(prob, precision=m.MM_FP32_DF64)
    d = torch.as_tensor(nb["d"], device="cuda")
    x1 = torch.empty(op.n_obs, 3, dtype=torch.float64, device="cuda")
    x2 = torch.empty_like(x1)
    m.mm_solve_tod(gp, d, x1, tol=cfg.tol, max_iter=5000, precision=m.MM_FP32)
    b = torch.empty_like(x1)
    m.mm_rhs(gp, d, b)
    m.mm_pcg_solve(gp, b, x2, tol=cfg.tol, max_iter=5000, precision=m.MM_FP32)
    assert rel(x1.cpu().numpy(), x2.cpu().numpy()) < 1e-5


def test_tod_solve_multi_rhs_and_fp64_fallback(tiny):
    """Two TOD columns on a mixed plan, and the FP64-class path (IEEE FP64 plan) through the same
    entry point."""
    cfg, prob, nb, op, ref = tiny
    m = mm()
    rng = np.random.default_rng(3)
    d2 = np.stack([nb["d"], nb["d"] + 0.1 * rng.standard_normal(nb["d"].size)])
    gp, _, _ = plans(prob, precision=m.MM_FP32_DF64)
    x = torch.empty(2, op.n_obs, 3, dtype=torch.float64, device="cuda")
    infos = m.mm_solve_tod(gp, torch.as_tensor(d2, device="cuda"), x, tol=cfg.tol, max_iter=5000,
                           precision=m.MM_FP32)
    for r in range(2):
        assert infos[r].status == 0 and infos[r].true_rel_res < cfg.tol
        rr = O.pcg(op, O.rhs(op, d2[r]), tol=cfg.tol, max_iter=5000)
        assert rel(x[r].cpu().numpy(), rr.x) < 1e-5
    g64, _, _ = plans(prob, precision=m.MM_FP64)
    x64 = torch.empty(op.n_obs, 3, dtype=torch.float64, device="cuda")
    info = m.mm_solve_tod(g64, torch.as_tensor(nb["d"], device="cuda"), x64, tol=cfg.tol, max_iter=5000)[0]
    assert info.status == 0 and abs(info.iters - ref.iters) <= 1
    assert rel(x64.cpu().numpy(), ref.x) < 1e-6


def test_tod_solve_from_host_tod(tiny):
    """A host TOD (pinned) is copied to the plan and gives the same map as the device TOD."""
    cfg, prob, nb, op, ref = tiny
    m = mm()
    gp, _, _ = plans(prob, precision=m.MM_FP32_DF64)
    x1 = torch.empty(op.n_obs, 3, dtype=torch.float64, device="cuda")
    x2 = torch.empty_like(x1)
    m.mm_solve_tod(gp, torch.as_tensor(nb["d"], device="cuda"), x1, tol=cfg.tol, max_iter=5000, precision=m.MM_FP32)
    info = m.mm_solve_tod(gp, torch.as_tensor(nb["d"]).pin_memory(), x2, tol=cfg.tol, max_iter=5000,
                          precision=m.MM_FP32)[0]
    assert info.status == 0 and info.true_rel_res < cfg.tol
    assert rel(x2.cpu().numpy(), x1.cpu().numpy()) < 1e-6
