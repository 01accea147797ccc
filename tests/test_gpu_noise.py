"""Noise weights estimated from the data on the GPU (mm_estimate_bands) against the FP64 oracle
(periodogram, PSD fit, inverse band).  The GPU transforms are FP32 and the fit sums FP32 terms in
FP64, so the fitted parameters agree with the oracle's to ~1e-5 and the band, which the FP32 FFT
produces from them, to ~1e-5 of its largest coefficient; the tolerances below leave a factor of
ten on that."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import synth
from gpu_helpers import cuda, mm

pytestmark = pytest.mark.gpu


def blocks(seed=0):
    # 1/f blocks of several shapes: 4 full segments; 3 segments and a dropped partial one; a block
    # shorter than a segment (zero-padded); an empty block; a white-noise block
    g = torch.Generator().manual_seed(seed)
    lens = [4 * O.NOISE_SEG, 3 * O.NOISE_SEG + 5000, 20000, 0, 2 * O.NOISE_SEG]
    pars = [(1.1, 1.0, 1.5), (0.9, 0.3, 1.2), (1.0, 2.0, 2.0), (1.0, 1.0, 1.0), (1.3, 0.0, 1.0)]
    d = np.concatenate([synth.noise_block(n, 100.0, s, fk, a, g).numpy() if n else np.zeros(0)
                        for n, (s, fk, a) in zip(lens, pars)])
    pix = np.zeros(d.size, np.int32)
    rng = np.random.default_rng(seed)
    pix[rng.random(d.size) < 0.03] = -1            # scattered flags
    pix[1000:3000] = -1                            # and a run
    return lens, pix, d


def log_cost(P, theta):
    # the oracle's objective: sum over k >= 1 of (log P_k - log P(f_k; theta))^2, in FP64
    f = np.arange(1, P.size) / O.NOISE_SEG
    return float(np.sum((np.log(P[1:]) - np.log(O.psd_model(f, theta))) ** 2))


@pytest.mark.parametrize("lam", [1024, 8192])
def test_estimated_bands_match_oracle(lam):
    lens, pix, d = blocks()
    bands, par = mm().mm_estimate_bands(len(lens), 1, lens, cuda(pix).to(torch.int32), cuda(d), lam)
    ob, oth = O.estimate_bands(d, pix, lens, lam)
    P, _ = O.periodogram(d, pix, lens)
    g = bands.cpu().numpy()
    for b, n in enumerate(lens):
        if n == 0:
            assert np.all(par[b] == 0) and np.all(g[b] == 0)
            continue
        # every fit is as good as the oracle's in the oracle's own objective.  White noise (block 4)
        # has no minimiser: the cost decreases along a valley (alpha -> 0, f_knee -> infinity)
        # where either optimiser may stop, so there the bound is 1e-3 of the cost (a difference of
        # ~10 in a sum of 16384 squared log-residuals, far below the periodogram's noise)
        rel = 1e-3 if b == 4 else 1e-6
        assert log_cost(P[b], par[b]) <= log_cost(P[b], oth[b]) * (1 + rel) + 1e-9, b
        if b != 4:   # blocks with a 1/f excess: the minimiser is unique
            assert np.max(np.abs(par[b] - oth[b])) < 1e-4, (b, par[b], oth[b])
            assert np.max(np.abs(g[b] - ob[b])) <= 1e-4 * np.max(np.abs(ob[b])), b
        # the inverse transform alone, from the GPU's own parameters
        ref = O.band_from_psd(par[b], lam)
        assert np.max(np.abs(g[b] - ref)) <= 1e-4 * np.max(np.abs(ref)), b


def test_fully_flagged_block_gives_zeros():
    lens, pix, d = blocks(1)
    off = np.concatenate([[0], np.cumsum(lens)])
    pix[off[1]:off[2]] = -1
    bands, par = mm().mm_estimate_bands(len(lens), 1, lens, cuda(pix).to(torch.int32), cuda(d), 512)
    assert np.all(par[1] == 0) and float(bands[1].abs().max()) == 0.0


def test_estimated_bands_drive_a_solve():
    # plan and solve with the weights estimated on the GPU; the oracle solves with the same weights
    cfg = synth.tiny_config()
    prob = synth.make_ground_problem(cfg)
    nb = synth.to_numpy(prob)
    bands, _ = mm().mm_estimate_bands(prob.n_det, prob.n_int, nb["block_len"].tolist(), prob.pix.cuda(),
                                      prob.d.cuda(), prob.lam)
    plan = mm().mm_plan(prob.n_det, prob.n_int, nb["block_len"].tolist(), prob.n_pix, prob.pix.cuda(),
                        prob.psi.cuda(), prob.lam, bands, precision=3)
    op = O.make_plan(nb["pix"], nb["psi"], nb["block_len"], bands.cpu().numpy(), nb["n_pix"])
    assert plan.n_obs == op.n_obs
    b = torch.empty(op.n_obs, 3, dtype=torch.float64, device="cuda")
    mm().mm_rhs(plan, prob.d.cuda(), b)
    bo = O.rhs(op, nb["d"])
    assert np.max(np.abs(b.cpu().numpy() - bo)) <= 1e-11 * np.max(np.abs(bo))
    x = torch.empty_like(b)
    info = mm().mm_pcg_solve(plan, b, x, tol=1e-8, precision=1)[0]
    ref = O.pcg(op, bo, tol=1e-8)
    assert info.status == 0 and ref.converged
    assert np.linalg.norm(x.cpu().numpy() - ref.x) <= 1e-5 * np.linalg.norm(ref.x)


def test_estimate_bands_rejects_bad_lambda():
    lens, pix, d = blocks(2)
    with pytest.raises(mm().MMError) as ei:
        mm().mm_estimate_bands(len(lens), 1, lens, cuda(pix).to(torch.int32), cuda(d), 12289)
    assert ei.value.code == 1
