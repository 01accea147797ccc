"""Template map-making (diagonal weights, F_T = W - W T (T^T W T)^+ T^T W; Appendix A templates) on the
GPU against the FP64 oracle.  The FP64 operator agrees with the oracle to rounding (1e-11); the FP32
one filters in FP32 (2e-5, as the other FP32 operators)."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from gpu_helpers import cuda, mm, plans, rel_max

pytestmark = pytest.mark.gpu


def problem(seed=61, lens=(30000, 1, 0, 17000, 25003), n_pix=200):
    prob = synth.random_problem(len(lens), list(lens), n_pix, 0, seed, gap_frac=0.04, hits_per_pix_min=8)
    rng = np.random.default_rng(seed)
    w = 0.5 + rng.random(len(lens))
    prob.band = torch.as_tensor(w[:, None])
    n = int(np.sum(lens))
    az = np.concatenate([np.abs(np.sin(np.linspace(0, 9, m))) * 10 + rng.normal(0, 0.01, m) if m else np.zeros(0)
                         for m in lens]).astype(np.float32)
    hwp = ((2 * np.pi * 0.37 * np.arange(n)) % (2 * np.pi)).astype(np.float32)
    return prob, w, az, hwp


def attach(gp, tm, az, hwp):
    mm().mm_templates_set(gp, n_poly=tm.n_poly, n_az=tm.n_az, n_hwp=tm.n_hwp, az_interp=tm.interp,
                          az=torch.as_tensor(az, device="cuda"), hwp=torch.as_tensor(hwp, device="cuda"))


# the mixes cover every kernel instantiation (<4,4>, <4,8>, <16,8>), binned and interpolated azimuth,
# azimuth only, and more dense (Legendre, HWP) pairs than setup threads (16 + 2 x 8 columns: 528 pairs)
TMS = [O.Templates(n_poly=3, n_az=6, n_hwp=2), O.Templates(n_poly=2, n_az=5, n_hwp=1, interp=True),
       O.Templates(n_poly=16), O.Templates(n_az=64), O.Templates(n_hwp=8, n_poly=4, n_az=30),
       O.Templates(n_poly=16, n_hwp=8)]


@pytest.mark.parametrize("ti", range(len(TMS)))
@pytest.mark.parametrize("precision,tol", [(0, 1e-11), (2, 1e-11), (1, 2e-5)])
def test_template_apply_matches_oracle(ti, precision, tol):
    tm = TMS[ti]
    prob, w, az, hwp = problem()
    gp, op, nb = plans(prob, precision=precision)
    attach(gp, tm, az, hwp)
    x = np.random.default_rng(ti).standard_normal((op.n_obs, 3))
    y = torch.empty(op.n_obs, 3, dtype=torch.float64, device="cuda")
    mm().mm_apply_A(gp, cuda(x), y)
    assert rel_max(y.cpu().numpy(), O.apply_A_templates(op, w, tm, az, hwp, x)) < tol


@pytest.mark.parametrize("fp32_d", [False, True])
def test_template_rhs_matches_oracle(fp32_d):
    tm = TMS[0]
    prob, w, az, hwp = problem(62)
    gp, op, nb = plans(prob, precision=3)
    attach(gp, tm, az, hwp)
    d = nb["d"].astype(np.float32) if fp32_d else nb["d"]
    b = torch.empty(op.n_obs, 3, dtype=torch.float64, device="cuda")
    mm().mm_rhs(gp, torch.as_tensor(d, device="cuda"), b)
    assert rel_max(b.cpu().numpy(), O.rhs_templates(op, w, tm, az, hwp, d.astype(np.float64))) < 1e-11


@pytest.mark.parametrize("precision", [0, 1])
def test_template_solve_removes_template_signals(precision):
    # d = P m + template signals with large amplitudes (no noise): the solve recovers Q, U and I up
    # to its mean (degenerate with the constant templates)
    tm = O.Templates(n_poly=2, n_az=8, n_hwp=2)
    prob, w, az, hwp = problem(63, lens=(40000, 30000, 35000), n_pix=100)
    nb = synth.to_numpy(prob)
    op = O.make_plan(nb["pix"], nb["psi"], nb["block_len"], w[:, None], nb["n_pix"])
    rng = np.random.default_rng(4)
    m = rng.standard_normal((op.n_obs, 3))
    d = O.unpoint(op, m)
    for b in range(3):
        lo, hi = op.offsets[b], op.offsets[b + 1]
        T = O.template_matrix(int(hi - lo), az[lo:hi], hwp[lo:hi], op.lpix[lo:hi] >= 0, tm)
        d[lo:hi] += T @ (rng.standard_normal(tm.k) * 20)
    gp, _, _ = plans(prob, precision=3)
    attach(gp, tm, az, hwp)
    b = torch.empty(op.n_obs, 3, dtype=torch.float64, device="cuda")
    mm().mm_rhs(gp, cuda(d), b)
    x = torch.empty_like(b)
    info = mm().mm_pcg_solve(gp, b, x, tol=1e-10, max_iter=3000, precision=precision)[0]
    assert info.status == 0
    xr = x.cpu().numpy()
    tolx = 1e-6 if precision == 0 else 1e-4
    assert np.max(np.abs(xr[:, 1:] - m[:, 1:])) < tolx
    assert np.max(np.abs((xr[:, 0] - xr[:, 0].mean()) - (m[:, 0] - m[:, 0].mean()))) < tolx


def test_templates_rejected_where_they_do_not_apply():
    prob, w, az, hwp = problem(64)
    gp, op, nb = plans(prob, precision=1)
    for kw in (dict(n_poly=17), dict(n_hwp=9), dict(n_poly=16, n_az=40, n_hwp=5), dict()):
        with pytest.raises(mm().MMError) as ei:
            mm().mm_templates_set(gp, az=torch.as_tensor(az, device="cuda"), hwp=torch.as_tensor(hwp, device="cuda"), **kw)
        assert ei.value.code == 1
    attach(gp, TMS[0], az, hwp)
    x = cuda(np.ones((op.n_obs, 3)))
    with pytest.raises(mm().MMError):
        mm().mm_apply_A_noalloc(gp, x, torch.empty_like(x))
    band_prob = synth.random_problem(2, [5000, 5000], 50, 16, 3, hits_per_pix_min=8)   # lambda = 16
    gp2, _, _ = plans(band_prob)
    with pytest.raises(mm().MMError) as ei:
        attach(gp2, TMS[0], np.zeros(10000, np.float32), np.zeros(10000, np.float32))
    assert ei.value.code == 1


@pytest.mark.parametrize("precision,tol", [(0, 1e-11), (2, 1e-11), (1, 2e-5)])
def test_template_apply_several_columns(precision, tol):
    # nrhs = 3 in one call (the block and enlarged solvers apply A to several columns at once):
    # every column equals the oracle's single-column operator
    tm = TMS[1]
    prob, w, az, hwp = problem(65)
    gp, op, nb = plans(prob, precision=precision)
    attach(gp, tm, az, hwp)
    X = np.random.default_rng(7).standard_normal((3, op.n_obs, 3))
    Y = torch.empty(3, op.n_obs, 3, dtype=torch.float64, device="cuda")
    mm().mm_apply_A(gp, cuda(X), Y)
    Yc = Y.cpu().numpy()
    for r in range(3):
        assert rel_max(Yc[r], O.apply_A_templates(op, w, tm, az, hwp, X[r])) < tol


def test_template_block_cg_matches_dense_solve():
    # block CG (mixed precision) on three right-hand sides of a template plan: the system is only
    # semi-definite (the I offset is free), so each column is compared with a least-squares solve
    # of the dense oracle system on Q, U, and its residual is checked with the oracle operator
    tm = O.Templates(n_poly=2, n_az=6, n_hwp=1)
    prob, w, az, hwp = problem(66, lens=(20000, 16000, 18000), n_pix=60)
    gp, op, nb = plans(prob, precision=3)
    attach(gp, tm, az, hwp)
    rng = np.random.default_rng(8)
    D = rng.standard_normal((3, op.lpix.size))
    B = np.stack([O.rhs_templates(op, w, tm, az, hwp, D[r]) for r in range(3)])
    A = np.stack([O.apply_A_templates(op, w, tm, az, hwp, e.reshape(-1, 3)).reshape(-1)
                  for e in np.eye(3 * op.n_obs)], axis=1)
    X = torch.empty(3, op.n_obs, 3, dtype=torch.float64, device="cuda")
    infos = mm().mm_block_cg_solve(gp, cuda(B), X, block_width=3, tol=1e-9, max_iter=3000)
    assert all(i.status == 0 for i in infos)
    Xc = X.cpu().numpy()
    for r in range(3):
        xs = np.linalg.lstsq(A, B[r].reshape(-1), rcond=None)[0].reshape(-1, 3)
        assert np.max(np.abs(Xc[r][:, 1:] - xs[:, 1:])) <= 1e-5 * np.max(np.abs(xs[:, 1:]))
        res = A @ Xc[r].reshape(-1) - B[r].reshape(-1)
        assert np.linalg.norm(res) <= 1e-8 * np.linalg.norm(B[r])


@pytest.mark.parametrize("variant", [0, 1])
def test_template_ecg_matches_dense_solve(variant):
    # enlarged CG (t = 4, FP32 search blocks) on a template plan, against a least-squares solve of
    # the dense oracle system on Q, U (the I offset is free)
    tm = O.Templates(n_poly=2, n_az=6, n_hwp=1)
    prob, w, az, hwp = problem(67, lens=(20000, 16000, 18000), n_pix=60)
    gp, op, nb = plans(prob, precision=3)
    attach(gp, tm, az, hwp)
    d = np.random.default_rng(9).standard_normal(op.lpix.size)
    b = O.rhs_templates(op, w, tm, az, hwp, d)
    A = np.stack([O.apply_A_templates(op, w, tm, az, hwp, e.reshape(-1, 3)).reshape(-1)
                  for e in np.eye(3 * op.n_obs)], axis=1)
    x = torch.empty(op.n_obs, 3, dtype=torch.float64, device="cuda")
    e = mm().mm_ecg_solve(gp, cuda(b), x, 4, variant=variant, tol=1e-9, max_iter=3000)
    assert e.status == 0
    xs = np.linalg.lstsq(A, b.reshape(-1), rcond=None)[0].reshape(-1, 3)
    xr = x.cpu().numpy()
    assert np.max(np.abs(xr[:, 1:] - xs[:, 1:])) <= 1e-5 * np.max(np.abs(xs[:, 1:]))
    assert np.linalg.norm(A @ xr.reshape(-1) - b.reshape(-1)) <= 1e-8 * np.linalg.norm(b)
