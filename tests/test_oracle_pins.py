"""Pins of the FP64 oracle to facts the paper and the mathematics fix (no GPU).

Each test is chosen so that a plausible slip in the oracle (a dropped term, a wrong sign, a wrong
factor in the angle, a transposed operand, wrap-around in the Toeplitz product) fails it.
"""
import math

import numpy as np
import pytest

import oracle as O
import synth


def tiny_problem(seed=0, n_blocks=3, block_len=(300, 170, 41), n_pix=40, lam=12, gap=0.05,
                 hits_min=6):
    p = synth.random_problem(n_blocks, list(block_len), n_pix, lam, seed, gap_frac=gap,
                             hits_per_pix_min=hits_min)
    return synth.to_numpy(p)


def plan_of(pb, **kw):
    return O.make_plan(pb["pix"], pb["psi"], pb["block_len"], pb["band"], pb["n_pix"], **kw)


# ---------------------------------------------------------------- pointing (Sect. 2 HWP model)

def test_weights_closed_form():
    psi = np.array([0.0, math.pi / 8, math.pi / 4, math.pi / 2, 3 * math.pi / 4], np.float32)
    w = O.pointing_weights(psi)
    h = math.sqrt(0.5)
    want = np.array([[1, 1, 0], [1, h, h], [1, 0, 1], [1, -1, 0], [1, 0, -1]], float)
    np.testing.assert_allclose(w, want, atol=2e-7)   # float32 angle rounding only


def test_unpoint_intensity_only_is_one():
    pb = tiny_problem()
    pl = plan_of(pb)
    m = np.zeros((pl.n_obs, 3))
    m[:, 0] = 1.0
    t = O.unpoint(pl, m)
    np.testing.assert_array_equal(t, np.where(pl.lpix >= 0, 1.0, 0.0))


def test_point_is_adjoint_of_unpoint():
    pb = tiny_problem(seed=3)
    pl = plan_of(pb)
    rng = np.random.default_rng(1)
    m = rng.standard_normal((pl.n_obs, 3))
    t = rng.standard_normal(pl.lpix.size)
    lhs = np.dot(O.unpoint(pl, m), t)
    rhs = np.vdot(m, O.point(pl, t))
    assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + np.linalg.norm(m) * np.linalg.norm(t))


def test_point_of_ones_gives_hits():
    pb = tiny_problem(seed=4)
    pl = plan_of(pb)
    out = O.point(pl, np.ones(pl.lpix.size))
    cnt = np.bincount(pl.lpix[pl.lpix >= 0], minlength=pl.n_obs)
    np.testing.assert_array_equal(out[:, 0], cnt)


# ---------------------------------------------------------------- Toeplitz (Eq. MADCAP, stbmm)

@pytest.mark.parametrize("lam", [0, 1, 5, 40, 400])
def test_toeplitz_direct_equals_dense(lam):
    rng = np.random.default_rng(lam)
    bl = np.array([37, 1, 200, 64])
    band = rng.standard_normal((bl.size, lam + 1))
    t = rng.standard_normal(bl.sum())
    y = O.toeplitz_direct(band, bl, t)
    off = O.block_offsets(bl)
    for b in range(bl.size):
        T = O.toeplitz_dense(band[b], bl[b])
        np.testing.assert_allclose(y[off[b]:off[b + 1]], T @ t[off[b]:off[b + 1]],
                                   rtol=0, atol=1e-12)


@pytest.mark.parametrize("lam", [0, 3, 64, 300])
def test_toeplitz_fft_equals_direct(lam):
    rng = np.random.default_rng(10 + lam)
    bl = np.array([1000, 5, 129, 2048])
    band = rng.standard_normal((bl.size, lam + 1))
    t = rng.standard_normal(bl.sum())
    y1 = O.toeplitz_direct(band, bl, t)
    y2 = O.toeplitz_fft(band, bl, t)
    assert np.max(np.abs(y1 - y2)) <= 1e-12 * np.max(np.abs(y1))


def test_toeplitz_no_wrap_no_cross_block():
    lam = 7
    bl = np.array([50, 50])
    band = np.tile(np.arange(1.0, lam + 2.0), (2, 1))
    t = np.zeros(100)
    t[50] = 1.0                      # first sample of block 1
    y = O.toeplitz_fft(band, bl, t)
    assert np.all(y[:50] == 0)       # nothing leaks into block 0
    np.testing.assert_allclose(y[50:50 + lam + 1], band[1], atol=1e-13)
    assert np.all(np.abs(y[50 + lam + 1:]) < 1e-13)   # and nothing wraps to the block's end


def test_toeplitz_white_band_is_scaled_identity():
    sig = 1.3
    c, _ = synth.inverse_noise_band(4096, 16, 100.0, sig, 0.0, 1.0)
    assert abs(float(c[0]) - 1 / sig ** 2) < 1e-14
    assert np.max(np.abs(c[1:].numpy())) < 1e-14
    t = np.random.default_rng(0).standard_normal(300)
    y = O.toeplitz_fft(c.numpy()[None, :], [300], t)
    np.testing.assert_allclose(y, t / sig ** 2, atol=1e-13)


# ---------------------------------------------------------------- BD block and excision (Sect. 2.4)

@pytest.mark.parametrize("n", [3, 4, 7, 16])
def test_bd_uniform_angles_cond_two(n):
    psi = (np.arange(n) * math.pi / n).astype(np.float32)   # 2psi uniform on [0, 2pi)
    c0 = 2.5
    band = np.array([[c0, 0.3, 0.1]])
    B, hits = O.bd_blocks(np.zeros(n, np.int32), psi, [n], band, 1)
    np.testing.assert_allclose(B[0], c0 * np.diag([n, n / 2, n / 2]), atol=1e-5)
    keep, cond = O.excise(B, hits)
    assert keep[0] and abs(cond[0] - 2.0) < 1e-5


def test_excision_rules():
    # pixel 0: 2 hits (excised); pixel 1: all samples at the same angle (singular, excised);
    # pixel 2: well sampled (kept)
    pix = np.array([0, 0, 1, 1, 1, 1, 2, 2, 2, 2], np.int32)
    psi = np.array([0, 1, .3, .3, .3, .3, 0, .4, .8, 1.2], np.float32)
    band = np.array([[1.0, 0.0]])
    B, hits = O.bd_blocks(pix, psi, [10], band, 3)
    keep, cond = O.excise(B, hits, 1e3)
    assert list(keep) == [False, False, True]
    pl = O.make_plan(pix, psi, [10], band, 3)
    assert pl.n_obs == 1 and list(pl.lpix) == [-1] * 6 + [0] * 4


def test_excision_cond_threshold_tie_kept():
    pix = np.zeros(4, np.int32)
    psi = (np.arange(4) * math.pi / 4).astype(np.float32)
    band = np.array([[1.0]])
    B, hits = O.bd_blocks(pix, psi, [4], band, 1)
    _, cond = O.excise(B, hits)
    keep, _ = O.excise(B, hits, cond_max=float(cond[0]))
    assert keep[0]
    keep, _ = O.excise(B, hits, cond_max=float(cond[0]) * (1 - 1e-9))
    assert not keep[0]


# ---------------------------------------------------------------- A = P^T N^-1 P (Sect. 3.2)

def test_apply_A_equals_dense_and_is_spd():
    pb = tiny_problem(seed=5)
    pl = plan_of(pb)
    A = O.dense_A(pl)
    rng = np.random.default_rng(2)
    x = rng.standard_normal((pl.n_obs, 3))
    np.testing.assert_allclose(O.apply_A(pl, x).reshape(-1), A @ x.reshape(-1),
                               rtol=0, atol=1e-11 * np.max(np.abs(A)) * np.abs(x).sum() / x.size
                               * 10)
    np.testing.assert_allclose(A, A.T, atol=1e-12 * np.max(np.abs(A)))
    assert np.linalg.eigvalsh(A).min() > 0


def test_apply_A_direct_and_fft_agree():
    pb = tiny_problem(seed=6, lam=60)
    p1 = plan_of(pb, toeplitz="direct")
    p2 = plan_of(pb, toeplitz="fft")
    x = np.random.default_rng(3).standard_normal((p1.n_obs, 3))
    y1, y2 = O.apply_A(p1, x), O.apply_A(p2, x)
    assert np.max(np.abs(y1 - y2)) <= 1e-12 * np.max(np.abs(y1))


def test_rhs_masks_gap_samples_of_d():
    pb = tiny_problem(seed=7)
    pl = plan_of(pb)
    d = pb["d"].copy()
    b1 = O.rhs(pl, d)
    d[pl.lpix < 0] = 1e6          # garbage at flagged/excised samples must not leak through N^-1
    b2 = O.rhs(pl, d)
    np.testing.assert_array_equal(b1, b2)


# ---------------------------------------------------------------- Algorithm 1 and special cases

def test_pcg_matches_dense_cholesky():
    pb = tiny_problem(seed=8)
    pl = plan_of(pb)
    b = O.rhs(pl, pb["d"])
    ms = O.dense_solve(pl, b)
    res = O.pcg(pl, b, tol=1e-12, max_iter=2000)
    assert res.converged
    assert np.linalg.norm(res.x - ms) <= 1e-9 * np.linalg.norm(ms)


def test_noiseless_recovers_sky():
    pb = tiny_problem(seed=9, lam=20)
    pl = plan_of(pb)
    m_true = np.random.default_rng(4).standard_normal((pl.n_obs, 3))
    d = O.unpoint(pl, m_true)
    res = O.pcg(pl, O.rhs(pl, d), tol=1e-13, max_iter=5000)
    assert np.linalg.norm(res.x - m_true) <= 1e-9 * np.linalg.norm(m_true)


def test_lambda_zero_one_iteration_binned_map():
    pb = tiny_problem(seed=10, lam=0)
    pl = plan_of(pb)
    b = O.rhs(pl, pb["d"])
    res = O.pcg(pl, b, tol=1e-10, max_iter=10)
    assert res.iters == 1
    np.testing.assert_allclose(res.x, O.binned_map(pl, pb["d"]), rtol=1e-10, atol=1e-12)


def test_pcg_history_monotone_in_A_norm_error():
    pb = tiny_problem(seed=11)
    pl = plan_of(pb)
    A = O.dense_A(pl)
    b = O.rhs(pl, pb["d"])
    ms = O.dense_solve(pl, b).reshape(-1)
    res = O.pcg(pl, b, tol=1e-10, max_iter=500, keep_iterates=True)
    errs = [float((x.reshape(-1) - ms) @ A @ (x.reshape(-1) - ms)) for x in res.iterates]
    assert all(e2 <= e1 * (1 + 1e-8) + 1e-24 for e1, e2 in zip(errs, errs[1:]))


# ---------------------------------------------------------------- Algorithm 2 (block, Orthomin)

def test_block_cg_s1_equals_pcg():
    pb = tiny_problem(seed=12)
    pl = plan_of(pb)
    b = O.rhs(pl, pb["d"])
    ref = O.pcg(pl, b, tol=1e-9, max_iter=500)
    blk = O.block_cg(pl, b[None], tol=1e-9, max_iter=500)
    assert blk.iters == ref.iters
    assert np.linalg.norm(blk.X[0] - ref.x) <= 1e-8 * np.linalg.norm(ref.x)


def test_block_cg_multi_rhs_columns_match_pcg():
    pb = tiny_problem(seed=13)
    pl = plan_of(pb)
    rng = np.random.default_rng(5)
    Bm = np.stack([O.rhs(pl, pb["d"] + rng.standard_normal(pb["d"].size)) for _ in range(4)])
    blk = O.block_cg(pl, Bm, tol=1e-10, max_iter=500)
    A = O.dense_A(pl)
    for j in range(4):
        xs = np.linalg.solve(A, Bm[j].reshape(-1))
        assert blk.converged[j]
        assert np.linalg.norm(blk.X[j].reshape(-1) - xs) <= 1e-7 * np.linalg.norm(xs)
    ref_iters = max(O.pcg(pl, Bm[j], tol=1e-10).iters for j in range(4))
    assert blk.iters <= ref_iters


# ---------------------------------------------------------------- Algorithm 3 and A-DEF1

def test_lanczos_relation():
    pb = tiny_problem(seed=14)
    pl = plan_of(pb)
    b = O.rhs(pl, pb["d"]).reshape(-1)
    m = 8
    T, V, AV, beta, vnext = O.lanczos(pl, b, m)
    A = O.dense_A(pl)
    np.testing.assert_allclose(AV, A @ V, atol=1e-10 * np.abs(A).max())
    em = np.zeros(m)
    em[-1] = 1
    resid = A @ V - V @ T - beta * np.outer(vnext, em)
    assert np.abs(resid).max() <= 1e-9 * np.abs(A).max()
    assert np.abs(V.T @ V - np.eye(m)).max() < 1e-6
    np.testing.assert_allclose(V[:, 0], b / np.linalg.norm(b), atol=1e-15)


def test_two_level_deflation_identities():
    pb = tiny_problem(seed=15)
    pl = plan_of(pb)
    b = O.rhs(pl, pb["d"])
    tl = O.two_level_from_lanczos(pl, b, 6)
    A = O.dense_A(pl)
    Z = tl.Z
    Q = Z @ tl.Einv @ Z.T
    lhs = (np.eye(A.shape[0]) - A @ Q) @ A @ Z            # (I - AQ) A Z = 0
    assert np.abs(lhs).max() <= 1e-8 * np.abs(A @ Z).max()
    for j in range(Z.shape[1]):                            # M_2lvl A Z = Z
        out = O.precond_2lvl(pl, tl, (A @ Z[:, j]).reshape(-1, 3)).reshape(-1)
        np.testing.assert_allclose(out, Z[:, j], atol=1e-8 * np.abs(Z[:, j]).max())


def test_two_level_never_more_iterations_than_bd():
    pb = tiny_problem(seed=16, n_pix=60, lam=30)
    pl = plan_of(pb)
    b = O.rhs(pl, pb["d"])
    bd = O.pcg(pl, b, tol=1e-8)
    tl = O.two_level_from_lanczos(pl, b, 8)
    two = O.pcg(pl, b, tol=1e-8, precond=lambda r: O.precond_2lvl(pl, tl, r))
    assert two.converged and two.iters <= bd.iters
    assert np.linalg.norm(two.x - bd.x) <= 1e-5 * np.linalg.norm(bd.x)


def test_apply_A_at_pixels_equals_apply_A():
    pb = tiny_problem(seed=17, lam=25)
    pl = plan_of(pb)
    rng = np.random.default_rng(8)
    xg = rng.standard_normal((pb["n_pix"], 3))
    full = O.apply_A(pl, xg[pl.obs_to_global])
    pixels = pl.obs_to_global[[0, 3, 7]]
    vals, scale = O.apply_A_at_pixels(pb["pix"], pb["psi"], pl.offsets, pb["band"], pl.keep, xg, pixels)
    np.testing.assert_allclose(vals, full[[0, 3, 7]], rtol=1e-12, atol=1e-12 * scale.max())


# ---------------------------------------------------------------- enlarged CG (Sect. 3.2, ECG)

def test_ecg_split_sums_to_residual():
    b = np.random.default_rng(3).standard_normal((37, 3))
    for t in (1, 2, 5, 37):
        R = O.ecg_split(b, t)
        assert R.shape == (t, 37, 3)
        np.testing.assert_array_equal(R.sum(axis=0), b)
        owner = np.argmax(np.any(R != 0, axis=2), axis=0)       # each pixel lives in one column
        assert np.all(np.count_nonzero(np.any(R != 0, axis=2), axis=0) == 1)
        assert np.all(np.diff(owner) >= 0)                       # contiguous, ordered ranges


def test_ecg_t1_orthomin_equals_pcg_iterates():
    # with one column the enlarged recurrence is PCG: P_1 = z / sqrt(z^T A z) etc.
    pb = tiny_problem(seed=21)
    pl = plan_of(pb)
    b = O.rhs(pl, pb["d"])
    ref = O.pcg(pl, b, tol=1e-9, max_iter=500, keep_iterates=True)
    e = O.ecg(pl, b, 1, tol=1e-9, max_iter=500, keep_iterates=True)
    assert e.iters == ref.iters and e.converged
    for xe, xp in zip(e.iterates, ref.iterates):
        assert np.linalg.norm(xe - xp) <= 1e-9 * np.linalg.norm(ref.x)


@pytest.mark.parametrize("variant", ["orthomin", "orthodir"])
@pytest.mark.parametrize("t", [2, 4, 8])
def test_ecg_matches_dense_solve(variant, t):
    pb = tiny_problem(seed=22)
    pl = plan_of(pb)
    b = O.rhs(pl, pb["d"])
    xs = np.linalg.solve(O.dense_A(pl), b.reshape(-1))
    e = O.ecg(pl, b, t, tol=1e-12, max_iter=2000, variant=variant)
    assert e.converged
    assert np.linalg.norm(e.x.reshape(-1) - xs) <= 1e-9 * np.linalg.norm(xs)
    # the Galerkin condition of each step: the new residual block is orthogonal to P_k
    assert max(e.galerkin) <= 1e-9


def test_ecg_orthomin_and_orthodir_agree():
    # equivalent in exact arithmetic when Z^T A Z stays well conditioned (Sect. 3.2)
    pb = tiny_problem(seed=23)
    pl = plan_of(pb)
    b = O.rhs(pl, pb["d"])
    a = O.ecg(pl, b, 4, tol=1e-8, max_iter=500, variant="orthomin", keep_iterates=True)
    d = O.ecg(pl, b, 4, tol=1e-8, max_iter=500, variant="orthodir", keep_iterates=True)
    assert abs(a.iters - d.iters) <= 1
    for xa, xd in zip(a.iterates[:5], d.iterates[:5]):
        assert np.linalg.norm(xa - xd) <= 1e-7 * np.linalg.norm(a.x)


def test_ecg_enlarging_reduces_iterations():
    # the enlarged Krylov space deflates the t smallest eigenvalues (Eq. RateConvECG)
    pb = tiny_problem(seed=24, block_len=(900, 700, 400), n_pix=60, lam=40)
    pl = plan_of(pb)
    b = O.rhs(pl, pb["d"])
    its = [O.ecg(pl, b, t, tol=1e-8, max_iter=2000).iters for t in (1, 2, 4, 8)]
    assert its[3] < its[0], its
    assert all(its[i + 1] <= its[i] + 1 for i in range(3)), its


# ---------------------------------------------------------------- 2lvl a priori (Sect. 3.2)

def test_two_level_apriori_columns_by_counting():
    # three blocks of one detector = three time intervals; count the kept hits by hand
    pb = tiny_problem(seed=31)
    pl = plan_of(pb)
    tl = O.two_level_apriori(pl, 3)
    n = pl.n_obs
    Z = tl.Z.reshape(n, 3, 3)
    counts = np.zeros((n, 3))
    for b in range(3):
        for t in range(pl.offsets[b], pl.offsets[b + 1]):
            if pl.lpix[t] >= 0:
                counts[pl.lpix[t], b] += 1
    np.testing.assert_allclose(Z[:, 0, :], counts / counts.sum(axis=1, keepdims=True), rtol=0, atol=1e-15)
    np.testing.assert_array_equal(Z[:, 1:, :], 0.0)                 # Q and U rows are zero
    np.testing.assert_allclose(Z[:, 0, :].sum(axis=1), 1.0, atol=1e-14)   # partition of unity
    one = O.two_level_apriori(pl, 1)                                 # a single interval: Z = 1 on I
    np.testing.assert_allclose(one.Z.reshape(n, 3)[:, 0], 1.0, atol=1e-15)


def test_two_level_apriori_deflation_identities_and_iterations():
    pb = tiny_problem(seed=32, n_pix=60, lam=30)
    pl = plan_of(pb)
    tl = O.two_level_apriori(pl, 3)
    A = O.dense_A(pl)
    Z = tl.Z
    Q = Z @ tl.Einv @ Z.T
    lhs = (np.eye(A.shape[0]) - A @ Q) @ A @ Z
    assert np.abs(lhs).max() <= 1e-8 * np.abs(A @ Z).max()
    for j in range(Z.shape[1]):
        out = O.precond_2lvl(pl, tl, (A @ Z[:, j]).reshape(-1, 3)).reshape(-1)
        np.testing.assert_allclose(out, Z[:, j], atol=1e-8 * np.abs(Z[:, j]).max())
    b = O.rhs(pl, pb["d"])
    bd = O.pcg(pl, b, tol=1e-8)
    two = O.pcg(pl, b, tol=1e-8, precond=lambda r: O.precond_2lvl(pl, tl, r))
    assert two.converged and two.iters <= bd.iters + 1
    assert np.linalg.norm(two.x - bd.x) <= 1e-6 * np.linalg.norm(bd.x)


# ---------------------------------------------------------------- noise weights from the data

def test_periodogram_parseval_and_white_level():
    rng = np.random.default_rng(41)
    seg = 256
    d = rng.standard_normal(seg) * 1.7
    P, nseg = O.periodogram(d, np.zeros(seg, np.int32), [seg], seg=seg)
    w = np.full(seg // 2 + 1, 2.0)
    w[0] = w[-1] = 1.0
    # one-sided Parseval: sum_k w_k |X_k|^2 = seg sum_t d_t^2, and P_k = |X_k|^2 / seg here
    assert nseg[0] == 1
    np.testing.assert_allclose(np.sum(w * P[0]), np.sum(d * d), rtol=1e-12)
    # white noise of variance s^2 averages to s^2 (64 segments)
    d = rng.standard_normal(64 * seg) * 1.3
    P, nseg = O.periodogram(d, np.zeros(d.size, np.int32), [d.size], seg=seg)
    assert nseg[0] == 64
    assert abs(np.mean(P[0, 1:-1]) / 1.69 - 1) < 0.02


def test_periodogram_cosine_and_gaps():
    seg, k0, amp = 512, 37, 0.8
    t = np.arange(2 * seg)
    d = amp * np.cos(2 * np.pi * k0 * t / seg)
    pix = np.zeros(t.size, np.int32)
    P, _ = O.periodogram(d, pix, [t.size], seg=seg)
    np.testing.assert_allclose(P[0, k0], amp ** 2 * seg / 4, rtol=1e-12)      # |X_k0| = amp seg / 2
    assert np.max(np.delete(P[0], k0)) < 1e-20 * P[0, k0]
    # flagged samples count neither as data nor in the normalisation
    pix[::2] = -1
    Pg, _ = O.periodogram(d, pix, [t.size], seg=seg)
    manual = np.zeros(seg // 2 + 1)
    for s_ in range(2):
        x = np.where(pix[s_ * seg:(s_ + 1) * seg] >= 0, d[s_ * seg:(s_ + 1) * seg], 0.0)
        manual += np.abs(np.fft.rfft(x)) ** 2 / (seg // 2)
    np.testing.assert_allclose(Pg[0], manual / 2, rtol=1e-12)


def test_fit_recovers_an_exact_model():
    seg = 4096
    theta = np.array([math.log(1.21), math.log(0.004), 1.7])
    f = np.arange(seg // 2 + 1) / seg
    P = np.zeros(f.size)
    P[1:] = O.psd_model(f[1:], theta)
    P[0] = P[1]
    np.testing.assert_allclose(O.fit_psd(P, seg), theta, rtol=1e-8, atol=1e-10)


def test_fit_of_a_noise_realisation():
    # 1/f noise with sigma 1.1, f_knee 1 Hz at 100 Hz, alpha 1.5, 32 segments
    g = __import__("torch").Generator().manual_seed(9)
    d = synth.noise_block(32 * O.NOISE_SEG, 100.0, 1.1, 1.0, 1.5, g).numpy()
    bands, th = O.estimate_bands(d, np.zeros(d.size, np.int32), [d.size], 1024)
    assert abs(math.exp(th[0, 0]) / 1.21 - 1) < 0.05
    assert abs(math.exp(th[0, 1]) / 0.01 - 1) < 0.25
    assert abs(th[0, 2] - 1.5) < 0.15
    # the band of the true PSD on the same grid and window: close to the estimated one
    true = O.band_from_psd(np.array([math.log(1.21), math.log(0.01), 1.5]), 1024)
    assert abs(bands[0, 0] / true[0] - 1) < 0.1


def test_band_from_psd_closed_forms():
    seg, lam = 64, 10
    # white PSD (f_knee -> 0) with 1/P(0) := 0: c_tau = (delta_tau - 1/seg) / sigma^2, windowed
    c = O.band_from_psd(np.array([math.log(2.0), -200.0, 1.0]), lam, seg)
    tau = np.arange(lam + 1)
    np.testing.assert_allclose(c, 0.5 * ((tau == 0) - 1.0 / seg) * np.exp(-0.5 * (tau / (lam / 2)) ** 2),
                               rtol=1e-12, atol=1e-15)
    # brute-force inverse DFT with explicit cosines and the Gaussian window
    theta = np.array([math.log(1.3), math.log(0.05), 1.2])
    f = np.arange(seg // 2 + 1) / seg
    S = np.zeros(f.size)
    S[1:] = 1.0 / O.psd_model(f[1:], theta)
    full = np.concatenate([S, S[-2:0:-1]])
    ref = np.array([sum(full[k] * math.cos(2 * math.pi * k * t / seg) for k in range(seg)) / seg
                    * math.exp(-0.5 * (t / (lam / 2)) ** 2) for t in range(lam + 1)])
    np.testing.assert_allclose(O.band_from_psd(theta, lam, seg), ref, rtol=1e-12, atol=1e-15)


# ---------------------------------------------------------------- template map-making (Appendix A)

def tmpl_problem(seed=51, lens=(3000, 2500, 0, 1700), n_pix=50):
    p = synth.random_problem(len(lens), list(lens), n_pix, 0, seed, gap_frac=0.05, hits_per_pix_min=6)
    nb = synth.to_numpy(p)
    rng = np.random.default_rng(seed)
    n = int(np.sum(lens))
    az = np.concatenate([np.abs(np.sin(np.linspace(0, 9, m))) * 10 + rng.normal(0, 0.01, m) for m in lens]) if n else np.zeros(0)
    hwp = (2 * np.pi * 0.37 * np.arange(n)) % (2 * np.pi)
    w = 0.5 + rng.random(len(lens))
    band = w[:, None]                                  # lambda = 0: c_0 = w_b (diagonal weights)
    pl = O.make_plan(nb["pix"], nb["psi"], nb["block_len"], band, nb["n_pix"])
    return pl, nb, w, az.astype(np.float32), hwp.astype(np.float32)


@pytest.mark.parametrize("interp", [False, True])
def test_template_filter_annihilates_templates_and_is_symmetric(interp):
    pl, nb, w, az, hwp = tmpl_problem()
    tm = O.Templates(n_poly=3, n_az=5, n_hwp=2, interp=interp)
    rng = np.random.default_rng(1)
    for b in (0, 1, 3):
        lo, hi = pl.offsets[b], pl.offsets[b + 1]
        kept = pl.lpix[lo:hi] >= 0
        T = O.template_matrix(int(hi - lo), az[lo:hi], hwp[lo:hi], kept, tm)
        for j in range(T.shape[1]):                     # F_T T = 0
            v = np.zeros(pl.lpix.size)
            v[lo:hi] = T[:, j]
            out = O.template_filter(pl, w, tm, az, hwp, v)
            assert np.max(np.abs(out)) <= 1e-10 * np.max(np.abs(w[b] * T[:, j]))
    u, v = rng.standard_normal((2, pl.lpix.size))     # <u, F v> = <F u, v>, <v, F v> >= 0
    Fu, Fv = O.template_filter(pl, w, tm, az, hwp, u), O.template_filter(pl, w, tm, az, hwp, v)
    assert abs(np.dot(u, Fv) - np.dot(Fu, v)) <= 1e-11 * np.linalg.norm(u) * np.linalg.norm(Fv)
    assert np.dot(v, Fv) >= -1e-12 * np.dot(v, v)


def test_template_columns_by_definition():
    n = 200
    az = np.linspace(3.0, 7.0, n)
    hwp = np.linspace(0.0, 12.0, n)
    kept = np.ones(n, bool)
    T = O.template_matrix(n, az, hwp, kept, O.Templates(n_poly=3, n_az=4, n_hwp=1))
    x = 2 * np.arange(n) / (n - 1) - 1
    np.testing.assert_allclose(T[:, 0], math.sqrt(1 / n), rtol=1e-15)
    np.testing.assert_allclose(T[:, 1], x * math.sqrt(3 / n), rtol=1e-12)
    np.testing.assert_allclose(T[:, 2], 0.5 * (3 * x * x - 1) * math.sqrt(5 / n), rtol=1e-12, atol=1e-15)
    bins = T[:, 3:7]
    np.testing.assert_array_equal(bins.sum(axis=1), 1.0)                        # one bin per sample
    np.testing.assert_array_equal(np.argmax(bins, axis=1), np.minimum(((az - 3) / 4 * 4).astype(int), 3))
    np.testing.assert_allclose(T[:, 7], np.cos(hwp), rtol=1e-15)
    np.testing.assert_allclose(T[:, 8], np.sin(hwp), rtol=1e-15, atol=1e-15)
    Ti = O.template_matrix(n, az, hwp, kept, O.Templates(n_az=5, interp=True))
    np.testing.assert_allclose(Ti.sum(axis=1), 1.0, rtol=1e-14)                 # partition of unity
    np.testing.assert_allclose(Ti @ np.linspace(3, 7, 5), az, rtol=1e-13)      # reproduces linear az
    assert np.all(np.count_nonzero(Ti, axis=1) <= 2)


def test_no_templates_is_the_diagonal_weighted_operator():
    pl, nb, w, az, hwp = tmpl_problem(seed=52)
    x = np.random.default_rng(2).standard_normal((pl.n_obs, 3))
    np.testing.assert_allclose(O.apply_A_templates(pl, w, O.Templates(), az, hwp, x), O.apply_A(pl, x),
                               rtol=1e-12, atol=1e-12)


def test_templates_remove_a_template_signal_from_the_map():
    # d = P m + sum of template signals (no noise): the template map-maker recovers m exactly,
    # the diagonal-weighted (binned) solution does not
    pl, nb, w, az, hwp = tmpl_problem(seed=53, lens=(6000, 5000, 4000), n_pix=30)
    tm = O.Templates(n_poly=2, n_az=4, n_hwp=2)
    rng = np.random.default_rng(3)
    m = rng.standard_normal((pl.n_obs, 3))
    d = O.unpoint(pl, m)
    for b in range(3):
        lo, hi = pl.offsets[b], pl.offsets[b + 1]
        T = O.template_matrix(int(hi - lo), az[lo:hi], hwp[lo:hi], pl.lpix[lo:hi] >= 0, tm)
        d[lo:hi] += T @ (rng.standard_normal(tm.k) * 5)
    A = np.stack([O.apply_A_templates(pl, w, tm, az, hwp, e.reshape(-1, 3)).reshape(-1)
                  for e in np.eye(3 * pl.n_obs)], axis=1)
    b = O.rhs_templates(pl, w, tm, az, hwp, d).reshape(-1)
    x = np.linalg.lstsq(A, b, rcond=None)[0].reshape(-1, 3)
    # the total-intensity offset is degenerate with the constant templates: compare Q, U and the
    # I map up to its mean
    np.testing.assert_allclose(x[:, 1:], m[:, 1:], atol=1e-8)
    np.testing.assert_allclose(x[:, 0] - x[:, 0].mean(), m[:, 0] - m[:, 0].mean(), atol=1e-8)
    xb = O.pcg(pl, O.rhs(pl, d), tol=1e-12).x
    assert np.max(np.abs(xb[:, 1:] - m[:, 1:])) > 1e-3
