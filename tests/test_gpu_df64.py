"""Parity of the double-float (df64) FP64-class operators with the FP64 oracle.

Plans of precision MM_DF64 run every FP64-class tile (A-application, right-hand side) in
double-float arithmetic on the FP32 pipes; MM_FP32_DF64 plans run the CG iterations in FP32 and the
right-hand side, residual replacement and true residual in df64.  A df64 value carries a 48-bit
significand, so the overlap-save FFT's normwise error is ~2^-47 log2(L) ~ 1e-13 of the band's
dynamic range: the FP64 tolerance of the other parity tests (1e-11) applies unchanged.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from gpu_helpers import cuda, mm, plans, rel_max

pytestmark = pytest.mark.gpu

DF64, FP32_DF64 = 2, 3


def small(seed=0, block_len=(70001, 5, 33000, 12, 0, 40000), n_pix=300, lam=1024, gap=0.02):
    return synth.random_problem(len(block_len), list(block_len), n_pix, lam, seed, gap_frac=gap,
                                hits_per_pix_min=4)


@pytest.mark.parametrize("seed,lam", [(5, 1024), (11, 12288), (12, 7)])
def test_apply_A_df64_matches_oracle(seed, lam):
    prob = small(seed, lam=lam)
    gp, op, _ = plans(prob, precision=DF64)
    x = np.random.default_rng(seed).standard_normal((op.n_obs, 3))
    y = torch.empty(op.n_obs, 3, dtype=torch.float64, device="cuda")
    mm().mm_apply_A(gp, cuda(x), y)
    assert rel_max(y.cpu().numpy(), O.apply_A(op, x)) < 1e-11


def test_apply_A_df64_multi_rhs():
    prob = small(7)
    gp, op, _ = plans(prob, precision=DF64)
    X = np.random.default_rng(7).standard_normal((3, op.n_obs, 3))
    Y = torch.empty(3, op.n_obs, 3, dtype=torch.float64, device="cuda")
    mm().mm_apply_A(gp, cuda(X), Y)
    for j in range(3):
        assert rel_max(Y[j].cpu().numpy(), O.apply_A(op, X[j])) < 1e-11


def test_apply_A_df64_close_to_fp64():
    # the df64 and IEEE FP64 operators agree far below the FP32 one's error
    prob = small(13)
    g64, op, _ = plans(prob, precision=0)
    gdf, _, _ = plans(prob, precision=DF64)
    x = cuda(np.random.default_rng(13).standard_normal((op.n_obs, 3)))
    y64 = torch.empty_like(x)
    ydf = torch.empty_like(x)
    mm().mm_apply_A(g64, x, y64)
    mm().mm_apply_A(gdf, x, ydf)
    assert rel_max(ydf.cpu().numpy(), y64.cpu().numpy()) < 1e-12


@pytest.mark.parametrize("fp32_d", [False, True])
@pytest.mark.parametrize("precision", [DF64, FP32_DF64])
def test_rhs_df64_matches_oracle(fp32_d, precision):
    prob = small(8)
    gp, op, nb = plans(prob, precision=precision)
    d = nb["d"].astype(np.float32) if fp32_d else nb["d"]
    b = torch.empty(op.n_obs, 3, dtype=torch.float64, device="cuda")
    mm().mm_rhs(gp, torch.as_tensor(d, device="cuda"), b)
    assert rel_max(b.cpu().numpy(), O.rhs(op, d.astype(np.float64))) < 1e-11


def test_rhs_df64_multi_rhs():
    prob = small(14)
    gp, op, nb = plans(prob, precision=DF64)
    rng = np.random.default_rng(14)
    D = np.stack([nb["d"], nb["d"] + rng.standard_normal(nb["d"].size)])
    B = torch.empty(2, op.n_obs, 3, dtype=torch.float64, device="cuda")
    mm().mm_rhs(gp, cuda(D), B)
    for j in range(2):
        assert rel_max(B[j].cpu().numpy(), O.rhs(op, D[j])) < 1e-11


@pytest.fixture(scope="module")
def tiny_cfg():
    cfg = synth.tiny_config()
    prob = synth.make_ground_problem(cfg)
    _, op, nb = plans(prob)
    b_or = O.rhs(op, nb["d"])
    ref = O.pcg(op, b_or, tol=cfg.tol, max_iter=5000)
    return cfg, prob, op, nb, b_or, ref


def test_pcg_df64_tiny_config_matches_oracle(tiny_cfg):
    cfg, prob, op, nb, b_or, ref = tiny_cfg
    gp, _, _ = plans(prob, precision=DF64)
    b = torch.empty(op.n_obs, 3, dtype=torch.float64, device="cuda")
    mm().mm_rhs(gp, torch.as_tensor(nb["d"], device="cuda"), b)
    assert rel_max(b.cpu().numpy(), b_or) < 1e-11
    x = torch.empty_like(b)
    info = mm().mm_pcg_solve(gp, b, x, tol=cfg.tol, max_iter=5000)[0]   # graph-captured iterations
    assert ref.converged and info.status == 0
    assert abs(info.iters - ref.iters) <= 1
    err = np.linalg.norm(x.cpu().numpy() - ref.x) / np.linalg.norm(ref.x)
    assert err <= 1e-6, err
    assert info.true_rel_res < 10 * cfg.tol


@pytest.mark.parametrize("profile", [0, 1])
def test_pcg_fp32_df64_mixed_matches_oracle(tiny_cfg, profile):
    cfg, prob, op, nb, b_or, ref = tiny_cfg
    gp, _, _ = plans(prob, precision=FP32_DF64)
    b = torch.empty(op.n_obs, 3, dtype=torch.float64, device="cuda")
    mm().mm_rhs(gp, torch.as_tensor(nb["d"], device="cuda"), b)
    assert rel_max(b.cpu().numpy(), b_or) < 1e-11
    x = torch.empty_like(b)
    info = mm().mm_pcg_solve(gp, b, x, tol=cfg.tol, max_iter=5000, precision=1, profile=profile)[0]
    assert info.status == 0
    assert info.true_rel_res < cfg.tol
    # the reported true residual is the oracle's ||b - A x|| / ||b|| at the returned x
    xr = x.cpu().numpy()
    tr = np.linalg.norm(b_or - O.apply_A(op, xr)) / np.linalg.norm(b_or)
    assert abs(tr - info.true_rel_res) <= 1e-3 * cfg.tol + 1e-12
    err = np.linalg.norm(xr - ref.x) / np.linalg.norm(ref.x)
    assert err <= 1e-5, err
