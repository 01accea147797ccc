"""Full-size parity on the ground workload (512 det x 4 int x 524,288 samples, lambda = 8192):
the plan and the A-applications (FP64, FP32 segment walker, df64) in the launch configuration the
benchmark times, checked on sampled output pixels that the oracle computes one by one.

The oracle's own excision decision (block-Jacobi blocks accumulated over all 1.07e9 samples,
hits >= 3 and cond <= 1e3) must equal the plan's compaction bit for bit; (A x)_p at a few random
pixels must match within the tolerances of the other parity tests, judged against the sum of the
absolute values of the terms of each output (cancellation makes a relative error meaningless).
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from gpu_helpers import cuda, mm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ground():
    cfg = synth.ground_config()
    prob = synth.make_ground_problem(cfg, device="cuda", with_noise=False, with_signal=False)
    pix = prob.pix.cpu().numpy()
    psi = prob.psi.cpu().numpy()
    band = prob.band.numpy()
    bl = prob.block_len.numpy()
    off = O.block_offsets(bl)
    # oracle excision over the whole data set, 64 blocks at a time
    B = np.zeros((cfg.n_pix, 3, 3))
    hits = np.zeros(cfg.n_pix, dtype=np.int64)
    step = 64
    for b0 in range(0, bl.size, step):
        b1 = min(b0 + step, bl.size)
        sl = slice(off[b0], off[b1])
        Bc, hc = O.bd_blocks(pix[sl], psi[sl], bl[b0:b1], band[b0:b1], cfg.n_pix)
        B += Bc
        hits += hc
    keep, _ = O.excise(B, hits, 1e3)
    return cfg, prob, pix, psi, band, off, keep


@pytest.mark.parametrize("precision,tol", [(0, 1e-11), (1, 2e-5), (2, 1e-11)])
def test_ground_full_size_sampled_outputs(ground, precision, tol):
    cfg, prob, pix, psi, band, off, keep = ground
    m = mm()
    plan = m.mm_plan(prob.n_det, prob.n_int, prob.block_len.tolist(), prob.n_pix, prob.pix,
                     prob.psi, prob.lam, prob.band.cuda(), precision=precision)
    o2g = plan.obs_to_global.cpu().numpy()
    np.testing.assert_array_equal(o2g, np.nonzero(keep)[0])
    rng = np.random.default_rng(7 + precision)
    xg = rng.standard_normal((cfg.n_pix, 3))
    x = cuda(xg[o2g])
    y = torch.empty_like(x)
    m.mm_apply_A(plan, x, y)
    pixels = rng.choice(o2g, 5, replace=False)
    idx = [torch.nonzero(prob.pix == int(p)).flatten().cpu().numpy() for p in pixels]
    vals, scale = O.apply_A_at_pixels(pix, psi, off, band, keep, xg, pixels, idx)
    got = y.cpu().numpy()[np.searchsorted(o2g, pixels)]
    err = np.abs(got - vals) / scale[:, None]
    assert err.max() <= tol, err.max()
    plan.destroy()
