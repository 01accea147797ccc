"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by element.

Tolerances (derived from the arithmetic of each path):
  FP64 operators: max-norm relative error <= 1e-11 (overlap-save FFT rounding ~ 1e-15 log2 L per
  sample, times the band's dynamic range; the direct sum is ~1e-15).
  FP32 operators: <= 2e-5 (float32 rounding of weights, map and a 15-pass FFT, ~ 1e-6 typical,
  with the band's dynamic range on top).
  Integer work (pixel compaction, excision): bit-exact.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from gpu_helpers import cuda, mm, plans, rel_max

pytestmark = pytest.mark.gpu


def small(seed=0, block_len=(70001, 5, 33000, 12, 0, 40000), n_pix=300, lam=1024, gap=0.02):
    return synth.random_problem(len(block_len), list(block_len), n_pix, lam, seed, gap_frac=gap,
                                hits_per_pix_min=4)


# ----------------------------------------------------------------------- plan (a1, a3)

@pytest.mark.parametrize("seed", [0, 1])
def test_compaction_and_bd_match_oracle(seed):
    prob = small(seed)
    # make a few pixels ill-conditioned: all samples of pixel 7 at one angle, pixel 9 with 2 hits
    pix = prob.pix.clone()
    psi = prob.psi.clone()
    psi[pix == 7] = 0.3
    pix[pix == 9] = 11
    idx = torch.nonzero(pix == 11)[:2, 0]
    pix[idx] = 9
    prob.pix, prob.psi = pix, psi
    gp, op, _ = plans(prob)
    assert gp.n_obs == op.n_obs
    np.testing.assert_array_equal(gp.obs_to_global.cpu().numpy(), op.obs_to_global)
    assert 7 not in set(op.obs_to_global) and 9 not in set(op.obs_to_global)
    # M_BD through mm_precond vs the oracle's inverse blocks
    r = np.random.default_rng(seed).standard_normal((op.n_obs, 3))
    z = torch.empty(op.n_obs, 3, dtype=torch.float64, device="cuda")
    mm().mm_precond(gp, cuda(r), z)
    assert rel_max(z.cpu().numpy(), O.precond_bd(op, r)) < 1e-12


def test_host_inputs_equal_device_inputs():
    prob = small(3)
    gd, op, _ = plans(prob, on_device=True)
    gh, _, _ = plans(prob, on_device=False)
    x = cuda(np.random.default_rng(0).standard_normal((op.n_obs, 3)))
    y1 = torch.empty_like(x)
    y2 = torch.empty_like(x)
    mm().mm_apply_A(gd, x, y1)
    mm().mm_apply_A(gh, x, y2)
    # same plan either way; only the order of the atomic scatter differs
    assert rel_max(y1.cpu().numpy(), y2.cpu().numpy()) < 1e-13


# ----------------------------------------------------------------------- P, N^-1, P^T (a5-a7)

@pytest.mark.parametrize("seed", [0, 2])
def test_unpoint_point_match_oracle(seed):
    prob = small(seed)
    gp, op, _ = plans(prob)
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((op.n_obs, 3))
    t = torch.empty(gp.n_samples, dtype=torch.float64, device="cuda")
    mm().mm_apply_P(gp, cuda(x), t)
    assert rel_max(t.cpu().numpy(), O.unpoint(op, x)) < 1e-14
    tt = rng.standard_normal(gp.n_samples)
    y = torch.empty(op.n_obs, 3, dtype=torch.float64, device="cuda")
    mm().mm_apply_Pt(gp, cuda(tt), y)
    assert rel_max(y.cpu().numpy(), O.point(op, tt)) < 1e-12


@pytest.mark.parametrize("lam", [0, 1, 17, 1024, 8192, 12288])
@pytest.mark.parametrize("algo", [1, 3])
def test_toeplitz_matches_definition(lam, algo):
    if algo == 3 and lam > 1024:
        pytest.skip("direct sum only for modest bands")
    prob = small(4, block_len=(70001, 3, 9000, 1, 40000), lam=lam)
    gp, op, nb = plans(prob, algo=algo)
    t = np.random.default_rng(lam).standard_normal(gp.n_samples)
    y = torch.empty_like(cuda(t))
    mm().mm_apply_Ninv(gp, cuda(t), y)
    ref = O.toeplitz_direct(nb["band"], nb["block_len"], t) if lam <= 64 else \
        O.toeplitz_fft(nb["band"], nb["block_len"], t)
    assert rel_max(y.cpu().numpy(), ref) < 1e-11


@pytest.mark.parametrize("algo", [1, 3])
def test_apply_A_fp64_matches_oracle(algo):
    prob = small(5)
    gp, op, _ = plans(prob, algo=algo)
    x = np.random.default_rng(5).standard_normal((op.n_obs, 3))
    y = torch.empty(op.n_obs, 3, dtype=torch.float64, device="cuda")
    mm().mm_apply_A(gp, cuda(x), y)
    assert rel_max(y.cpu().numpy(), O.apply_A(op, x)) < 1e-11


@pytest.mark.parametrize("tile_steps", [1, 2, 5])
def test_apply_A_fp32_matches_oracle(tile_steps):
    # blocks of 70001 / 33000 / 40000 samples span several tiles: tile_steps > 1 walks them with
    # the overlap kept in shared memory
    prob = small(6)
    gp, op, _ = plans(prob, precision=1, tile_steps=tile_steps)
    x = np.random.default_rng(6).standard_normal((op.n_obs, 3))
    y = torch.empty(op.n_obs, 3, dtype=torch.float64, device="cuda")
    mm().mm_apply_A(gp, cuda(x), y)
    assert rel_max(y.cpu().numpy(), O.apply_A(op, x)) < 2e-5


@pytest.mark.parametrize("lam", [6145, 8192, 12288])
def test_apply_A_fp32_large_lambda_matches_oracle(lam):
    """Above lambda = 6144 the FP32 operator can run N^-1 on 65536-sample tiles split over 2-CTA
    clusters (the autotuner times them against 32768-sample tiles): both on ragged blocks (shorter
    than one tile, one sample, empty), several columns."""
    prob = small(11, block_len=(150001, 1, 70000, 0, 40000), lam=lam)
    gp, op, _ = plans(prob, precision=3)
    rng = np.random.default_rng(lam)
    x = cuda(rng.standard_normal((2, op.n_obs, 3)))
    y = torch.empty_like(x)
    m = mm()
    m.mm_apply_A(gp, x, y)   # 32768-sample tiles
    for r in range(2):
        assert rel_max(y[r].cpu().numpy(), O.apply_A(op, x[r].cpu().numpy())) < 2e-5
    tune = m.mm_autotune(gp, max_width=1)   # times the 65536-sample 2-CTA tiles as a candidate
    assert tune["big_tiles"] in (0, 1) and tune["big_tiles_ms"] > 0
    assert tune["n_rejected"] == 0 and tune["max_rel_dev"] < 2e-5   # every candidate gave the same A x
    m.mm_apply_A(gp, x, y)
    for r in range(2):
        assert rel_max(y[r].cpu().numpy(), O.apply_A(op, x[r].cpu().numpy())) < 2e-5


@pytest.mark.parametrize("n_pix", [1, 7, 300])
@pytest.mark.parametrize("pt_sub", [4096, 8192, 16384])
def test_apply_A_fp32_segment_reduction_matches_oracle(n_pix, pt_sub):
    """The FP32 P^T by segment reduction over pixel-sorted sub-windows.  One or seven pixels make
    runs that span many threads' ranges (their partial sums meet in shared-memory atomics); 300
    pixels make short runs inside one range; ragged blocks (5, 12 samples, empty) and masked
    samples leave sub-windows partly empty.  A x within the FP32 tolerance of the oracle, for
    every sub-window size, several columns."""
    prob = small(13, block_len=(70001, 5, 33000, 12, 0, 9000), n_pix=n_pix, lam=256, gap=0.05)
    m = mm()
    gp, op, _ = plans(prob, precision=m.MM_FP32_DF64, pt_sub=pt_sub)
    rng = np.random.default_rng(n_pix)
    x = cuda(rng.standard_normal((2, op.n_obs, 3)))
    y = torch.empty_like(x)
    m.mm_apply_A(gp, x, y)
    for r in range(2):
        assert rel_max(y[r].cpu().numpy(), O.apply_A(op, x[r].cpu().numpy())) < 2e-5


def test_autotune_times_both_pt_forms():
    """mm_autotune times P^T by per-sample sums over the windows and by segment reduction (three
    sub-window sizes), checks each candidate's A x against the first's, keeps the fastest, and
    the tuned operator still matches the oracle."""
    prob = small(14, block_len=(70001, 5, 33000, 12, 0, 9000), n_pix=7, lam=256, gap=0.05)
    m = mm()
    gp, op, _ = plans(prob, precision=m.MM_FP32_DF64)
    tune = m.mm_autotune(gp, max_width=1)
    assert sorted(tune["seg_ms"]) == [0, 4096, 8192, 16384]
    assert tune["seg_ms"][tune["seg_sub"]] == min(tune["seg_ms"].values())
    assert tune["n_rejected"] == 0 and tune["max_rel_dev"] < 2e-5
    x = cuda(np.random.default_rng(3).standard_normal((op.n_obs, 3)))
    y = torch.empty_like(x)
    m.mm_apply_A(gp, x, y)
    assert rel_max(y.cpu().numpy(), O.apply_A(op, x.cpu().numpy())) < 2e-5


def test_apply_A_multi_rhs():
    prob = small(7)
    gp, op, _ = plans(prob)
    X = np.random.default_rng(7).standard_normal((3, op.n_obs, 3))
    Y = torch.empty(3, op.n_obs, 3, dtype=torch.float64, device="cuda")
    mm().mm_apply_A(gp, cuda(X), Y)
    for j in range(3):
        assert rel_max(Y[j].cpu().numpy(), O.apply_A(op, X[j])) < 1e-11


@pytest.mark.parametrize("fp32_d", [False, True])
def test_rhs_matches_oracle(fp32_d):
    prob = small(8)
    gp, op, nb = plans(prob)
    d = nb["d"].astype(np.float32) if fp32_d else nb["d"]
    b = torch.empty(op.n_obs, 3, dtype=torch.float64, device="cuda")
    dt = torch.as_tensor(d, device="cuda")
    mm().mm_rhs(gp, dt, b)
    assert rel_max(b.cpu().numpy(), O.rhs(op, d.astype(np.float64))) < 1e-11


@pytest.mark.parametrize("precision,algo", [(0, 0), (3, 0), (0, 3)])
@pytest.mark.parametrize("fp32_d", [False, True])
@pytest.mark.parametrize("pinned", [False, True])
def test_rhs_from_host_tod_matches_oracle(precision, algo, fp32_d, pinned):
    """The TOD may be handed over in host memory: the library stages it (IEEE FP64, double-float
    and direct-sum plans), two columns at once, and b matches the oracle's to the FP64 tolerance."""
    if algo == 3:
        prob = small(9, block_len=(7001, 5, 3300, 12, 0, 4000), lam=64)
    else:
        prob = small(9)
    gp, op, nb = plans(prob, precision=precision, algo=algo)
    rng = np.random.default_rng(5)
    d2 = np.stack([nb["d"], rng.standard_normal(nb["d"].size)])
    d2 = d2.astype(np.float32) if fp32_d else d2
    dh = torch.as_tensor(d2)
    if pinned:
        dh = dh.pin_memory()
    b = torch.empty(2, op.n_obs, 3, dtype=torch.float64, device="cuda")
    mm().mm_rhs(gp, dh, b)
    for r in range(2):
        assert rel_max(b[r].cpu().numpy(), O.rhs(op, d2[r].astype(np.float64))) < 1e-11


# ----------------------------------------------------------------------- PCG (a8, a11)

@pytest.fixture(scope="module")
def tiny_cfg():
    cfg = synth.tiny_config()
    prob = synth.make_ground_problem(cfg)
    gp, op, nb = plans(prob)
    b_or = O.rhs(op, nb["d"])
    ref = O.pcg(op, b_or, tol=cfg.tol, max_iter=5000)
    return cfg, prob, gp, op, nb, b_or, ref


def test_pcg_fp64_tiny_config_matches_oracle(tiny_cfg):
    cfg, prob, gp, op, nb, b_or, ref = tiny_cfg
    b = torch.empty(op.n_obs, 3, dtype=torch.float64, device="cuda")
    mm().mm_rhs(gp, torch.as_tensor(nb["d"], device="cuda"), b)
    assert rel_max(b.cpu().numpy(), b_or) < 1e-11
    x = torch.empty_like(b)
    info = mm().mm_pcg_solve(gp, b, x, tol=cfg.tol, max_iter=5000)[0]
    assert ref.converged and info.status == 0
    assert abs(info.iters - ref.iters) <= 1
    err = np.linalg.norm(x.cpu().numpy() - ref.x) / np.linalg.norm(ref.x)
    assert err <= 1e-6, err
    assert info.true_rel_res < 10 * cfg.tol


@pytest.mark.parametrize("tile_steps", [0, 3])
def test_pcg_fp32_mixed_tiny_config_matches_oracle(tiny_cfg, tile_steps):
    cfg, prob, gp, op, nb, b_or, ref = tiny_cfg
    if tile_steps:
        gp, _, _ = plans(prob, tile_steps=tile_steps)
    b = cuda(b_or)
    x = torch.empty_like(b)
    info = mm().mm_pcg_solve(gp, b, x, tol=cfg.tol, max_iter=5000, precision=1)[0]
    assert info.status == 0
    assert info.true_rel_res < cfg.tol
    # below the FP32 operator's accuracy the replacement restarts the recursion, so the mixed
    # solve needs only a few more iterations than the FP64 oracle (52 at 1e-8)
    assert info.iters <= ref.iters + 12, (info.iters, ref.iters)
    err = np.linalg.norm(x.cpu().numpy() - ref.x) / np.linalg.norm(ref.x)
    assert err <= 1e-5, err


def test_pcg_multi_rhs_columns_independent(tiny_cfg):
    cfg, prob, gp, op, nb, b_or, ref = tiny_cfg
    rng = np.random.default_rng(1)
    B = np.stack([b_or, O.rhs(op, nb["d"] + rng.standard_normal(nb["d"].size))])
    x = torch.empty(2, op.n_obs, 3, dtype=torch.float64, device="cuda")
    infos = mm().mm_pcg_solve(gp, cuda(B), x, tol=1e-7, max_iter=5000)
    for j in range(2):
        r = O.pcg(op, B[j], tol=1e-7, max_iter=5000)
        assert infos[j].status == 0 and abs(infos[j].iters - r.iters) <= 1
        assert np.linalg.norm(x[j].cpu().numpy() - r.x) <= 1e-6 * np.linalg.norm(r.x)


# ----------------------------------------------------------------------- special cases

def test_lambda_zero_converges_in_one_iteration():
    prob = small(9, lam=0)
    gp, op, nb = plans(prob)
    b = torch.empty(op.n_obs, 3, dtype=torch.float64, device="cuda")
    mm().mm_rhs(gp, torch.as_tensor(nb["d"], device="cuda"), b)
    x = torch.empty_like(b)
    info = mm().mm_pcg_solve(gp, b, x, tol=1e-10, max_iter=10)[0]
    assert info.iters == 1
    assert rel_max(x.cpu().numpy(), O.binned_map(op, nb["d"])) < 1e-10


def test_noiseless_map_recovered():
    prob = small(10, lam=300)
    gp, op, nb = plans(prob)
    m_true = np.random.default_rng(3).standard_normal((op.n_obs, 3))
    d = O.unpoint(op, m_true)
    b = torch.empty(op.n_obs, 3, dtype=torch.float64, device="cuda")
    mm().mm_rhs(gp, cuda(d), b)
    x = torch.empty_like(b)
    mm().mm_pcg_solve(gp, b, x, tol=1e-12, max_iter=5000)
    assert np.linalg.norm(x.cpu().numpy() - m_true) <= 1e-8 * np.linalg.norm(m_true)


def test_max_iter_returns_partial_and_enotconv():
    prob = small(11)
    gp, op, nb = plans(prob)
    b = cuda(O.rhs(op, nb["d"]))
    x = torch.empty_like(b)
    infos = mm().mm_pcg_solve(gp, b, x, tol=1e-14, max_iter=3, raise_on_error=False)
    assert infos[0].status == mm().MM_ENOTCONV and infos[0].iters == 3
    ref = O.pcg(op, O.rhs(op, nb["d"]), tol=1e-14, max_iter=3)
    assert rel_max(x.cpu().numpy(), ref.x) < 1e-9


def test_invalid_inputs_rejected():
    m = mm()
    prob = small(12)
    bad = prob.pix.clone()
    bad[5] = prob.n_pix
    with pytest.raises(m.MMError) as e:
        m.mm_plan(prob.n_det, 1, prob.block_len.tolist(), prob.n_pix, bad.cuda(), prob.psi.cuda(),
                  prob.lam, prob.band.cuda())
    assert e.value.code == m.MM_EINVAL
    with pytest.raises(m.MMError) as e:
        m.mm_plan(prob.n_det, 1, prob.block_len.tolist(), prob.n_pix, prob.pix.cuda(),
                  prob.psi.cuda(), 20000, torch.ones(prob.n_det, 20001, dtype=torch.float64).cuda())
    assert e.value.code == m.MM_EINVAL
    neg = prob.band.clone()
    neg[:, 1] = 0.9 * neg[:, 0]     # c0 + 2 c1 cos(w) < 0 near w = pi
    with pytest.raises(m.MMError) as e:
        m.mm_plan(prob.n_det, 1, prob.block_len.tolist(), prob.n_pix, prob.pix.cuda(),
                  prob.psi.cuda(), prob.lam, neg.cuda())
    assert e.value.code == m.MM_ENOTSPD
    allgap = torch.full_like(prob.pix, -1)
    with pytest.raises(m.MMError) as e:
        m.mm_plan(prob.n_det, 1, prob.block_len.tolist(), prob.n_pix, allgap.cuda(),
                  prob.psi.cuda(), prob.lam, prob.band.cuda())
    assert e.value.code == m.MM_ENOTSPD
    with pytest.raises(m.MMError) as e:   # not a sub-window size of the segment reduction
        m.mm_plan(prob.n_det, 1, prob.block_len.tolist(), prob.n_pix, prob.pix.cuda(),
                  prob.psi.cuda(), prob.lam, prob.band.cuda(), precision=m.MM_FP32, pt_sub=5000)
    assert e.value.code == m.MM_EINVAL


# ----------------------------------------------------------------------- arbitrary flag patterns

@pytest.mark.parametrize("precision,tol", [(0, 1e-11), (2, 1e-11), (1, 2e-5)])
def test_arbitrary_flag_patterns(precision, tol):
    # gapped Toeplitz (gstbmm, Sect. 3.1): half of the samples flagged at random, a whole block
    # flagged, and flags on the first and last samples of blocks; G on both sides of N^-1
    prob = small(10, block_len=(20000, 3000, 17000, 9), n_pix=200, lam=700, gap=0.5)
    pix = prob.pix.clone()
    off = np.concatenate([[0], np.cumsum(prob.block_len.numpy())])
    pix[off[1]:off[2]] = -1
    for b in range(4):
        if off[b + 1] > off[b]:
            pix[off[b]] = -1
            pix[off[b + 1] - 1] = -1
    prob.pix = pix
    gp, op, nb = plans(prob, precision=precision)
    x = np.random.default_rng(10).standard_normal((op.n_obs, 3))
    y = torch.empty(op.n_obs, 3, dtype=torch.float64, device="cuda")
    mm().mm_apply_A(gp, cuda(x), y)
    assert rel_max(y.cpu().numpy(), O.apply_A(op, x)) < tol
    b = torch.empty(op.n_obs, 3, dtype=torch.float64, device="cuda")
    mm().mm_rhs(gp, torch.as_tensor(nb["d"], device="cuda"), b)
    assert rel_max(b.cpu().numpy(), O.rhs(op, nb["d"])) < 1e-11   # the RHS runs FP64-class on every plan
