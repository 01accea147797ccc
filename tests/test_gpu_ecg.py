"""Enlarged CG (Sect. 3.2, ECG algorithm) through the C ABI against the FP64 oracle.

The GPU keeps the search blocks (Z, P, A P) in FP32 and X, R, the t x t matrices in FP64, as the
block CG does, so its recursive residual drifts from the true one at the ~1e-7 level; at the
tiny configuration's tolerance (1e-8) the solve then restarts from the FP64-class true residual,
which adds iterations.  Iteration counts are therefore bounded (no fewer than the oracle's minus
two, no more than twice the oracle's plus two); the answers are compared with the oracle's
solution (map error <= 1e-5, the mixed-precision bound) and the reported true residual with the
oracle's ||b - A x|| / ||b|| at the returned x.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from gpu_helpers import cuda, mm, plans

pytestmark = pytest.mark.gpu

ORTHOMIN, ORTHODIR = 0, 1


def small(seed=0, block_len=(70001, 5, 33000, 12, 0, 40000), n_pix=300, lam=1024, gap=0.02):
    return synth.random_problem(len(block_len), list(block_len), n_pix, lam, seed, gap_frac=gap,
                                hits_per_pix_min=4)


@pytest.fixture(scope="module")
def tiny():
    cfg = synth.tiny_config()
    prob = synth.make_ground_problem(cfg)
    gp, op, nb = plans(prob, precision=3)          # FP32 iterations, df64 true residual
    b = O.rhs(op, nb["d"])
    ref = O.pcg(op, b, tol=1e-10, max_iter=5000)
    return cfg, gp, op, b, ref


def true_rel(op, b, x):
    return np.linalg.norm(b - O.apply_A(op, x)) / np.linalg.norm(b)


@pytest.mark.parametrize("precision", [0, 1])
def test_ecg_t1_is_pcg(tiny, precision):
    cfg, gp, op, b, ref = tiny
    x = torch.empty(op.n_obs, 3, dtype=torch.float64, device="cuda")
    e = mm().mm_ecg_solve(gp, cuda(b), x, 1, tol=cfg.tol, precision=precision)
    p = O.pcg(op, b, tol=cfg.tol, max_iter=5000)
    assert e.status == 0 and p.iters - 2 <= e.iters <= 2 * p.iters + 2, (e.iters, p.iters)
    assert np.linalg.norm(x.cpu().numpy() - ref.x) <= 1e-5 * np.linalg.norm(ref.x)


@pytest.mark.parametrize("variant", [ORTHOMIN, ORTHODIR])
@pytest.mark.parametrize("t", [2, 8, 32])
@pytest.mark.parametrize("precision", [0, 1])
def test_ecg_matches_oracle(tiny, variant, t, precision):
    cfg, gp, op, b, ref = tiny
    x = torch.empty(op.n_obs, 3, dtype=torch.float64, device="cuda")
    e = mm().mm_ecg_solve(gp, cuda(b), x, t, variant=variant, tol=cfg.tol, precision=precision)
    o = O.ecg(op, b, t, tol=cfg.tol, max_iter=2000, variant=["orthomin", "orthodir"][variant])
    assert e.status == 0 and o.converged
    assert o.iters - 2 <= e.iters <= 2 * o.iters + 2, (e.iters, o.iters)
    xr = x.cpu().numpy()
    assert np.linalg.norm(xr - ref.x) <= 1e-5 * np.linalg.norm(ref.x)
    tr = true_rel(op, b, xr)
    assert e.true_rel_res < cfg.tol and tr < cfg.tol
    assert abs(tr - e.true_rel_res) <= 1e-3 * cfg.tol + 1e-13


def test_ecg_enlarging_reduces_iterations(tiny):
    cfg, gp, op, b, ref = tiny
    x = torch.empty(op.n_obs, 3, dtype=torch.float64, device="cuda")
    its = [mm().mm_ecg_solve(gp, cuda(b), x, t, tol=cfg.tol).iters for t in (1, 4, 16, 64)]
    assert its[-1] < its[0] and its[2] < its[0], its


def test_ecg_more_columns_than_pixels():
    # n_obs < t: some split columns are empty and their directions are dropped by the pivoted
    # Cholesky; the solve still reaches the oracle's answer
    prob = small(3, block_len=(9000, 7000), n_pix=20, lam=64)
    gp, op, nb = plans(prob, precision=3)
    assert op.n_obs < 64
    b = O.rhs(op, nb["d"])
    x = torch.empty(op.n_obs, 3, dtype=torch.float64, device="cuda")
    for variant in (ORTHOMIN, ORTHODIR):
        e = mm().mm_ecg_solve(gp, cuda(b), x, 64, variant=variant, tol=1e-9, precision=0)
        xs = np.linalg.solve(O.dense_A(op), b.reshape(-1)).reshape(-1, 3)
        assert e.status == 0
        assert np.linalg.norm(x.cpu().numpy() - xs) <= 1e-7 * np.linalg.norm(xs)


def test_ecg_ragged_blocks_df64_plan():
    # ragged blocks (incl. empty and 5-sample ones) on a df64 plan, FP64-class operator throughout
    prob = small(4)
    gp, op, nb = plans(prob, precision=2)
    b = O.rhs(op, nb["d"])
    ref = O.pcg(op, b, tol=1e-10, max_iter=5000)
    x = torch.empty(op.n_obs, 3, dtype=torch.float64, device="cuda")
    e = mm().mm_ecg_solve(gp, cuda(b), x, 8, variant=ORTHODIR, tol=1e-8, precision=0)
    assert e.status == 0
    assert np.linalg.norm(x.cpu().numpy() - ref.x) <= 1e-6 * np.linalg.norm(ref.x)


def test_ecg_zero_rhs_and_invalid_arguments(tiny):
    cfg, gp, op, b, ref = tiny
    x = torch.full((op.n_obs, 3), 7.0, dtype=torch.float64, device="cuda")
    e = mm().mm_ecg_solve(gp, torch.zeros_like(x), x, 4)
    assert e.status == 0 and e.iters == 0 and float(x.abs().max()) == 0.0
    for t, variant in ((0, 0), (65, 0), (4, 2)):
        with pytest.raises(mm().MMError) as ei:
            mm().mm_ecg_solve(gp, cuda(b), x, t, variant=variant)
        assert ei.value.code == 1
