"""Property-based pins of the oracle over random inputs (hypothesis; CPU only).  Each property
follows from the definitions, not from the oracle's own code paths:

* the FFT route of the banded Toeplitz product equals a dense matrix written from the band's
  definition (T_ij = c_|i-j| for |i - j| <= lambda, inside each block) for ragged blocks of any
  length, including blocks shorter than lambda and empty ones (Eq. MADCAP);
* A = P~^T N^-1 P~ is symmetric and positive definite on random ragged problems with gaps
  (Sect. 3.2);
* the template filter is a W-weighted projection: F_T W^+ F_T = F_T, with W^+ = 1/w on kept samples
  and 0 on masked ones; this holds for any template mix, because (T^T W T)^+ is a pseudo-inverse
  (Eq. genMapEstimator), and it fails for a misplaced weight or a wrong kernel inverse.
"""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import HealthCheck, assume, given, settings, strategies as st  # noqa: E402

import oracle as O  # noqa: E402
import synth  # noqa: E402

SETTINGS = settings(max_examples=25, deadline=None, suppress_health_check=[HealthCheck.too_slow])


@SETTINGS
@given(lens=st.lists(st.integers(min_value=0, max_value=300), min_size=1, max_size=4),
       lam=st.integers(min_value=0, max_value=40), seed=st.integers(min_value=0, max_value=2**31 - 1))
def test_toeplitz_fft_equals_dense_definition(lens, lam, seed):
    rng = np.random.default_rng(seed)
    band = rng.standard_normal((len(lens), lam + 1))
    t = rng.standard_normal(sum(lens))
    y = O.toeplitz_fft(band, lens, t)
    off = np.concatenate([[0], np.cumsum(lens)]).astype(int)
    for b, n in enumerate(lens):
        if n == 0:
            continue
        i = np.arange(n)
        dist = np.abs(i[:, None] - i[None, :])
        T = np.where(dist <= lam, band[b][np.minimum(dist, lam)], 0.0)
        ref = T @ t[off[b]:off[b + 1]]
        assert np.max(np.abs(y[off[b]:off[b + 1]] - ref)) <= 1e-11 * (np.abs(T).sum(axis=1).max() + 1.0)


@SETTINGS
@given(lens=st.lists(st.integers(min_value=40, max_value=500), min_size=1, max_size=3),
       lam=st.integers(min_value=0, max_value=24), gap=st.sampled_from([0.0, 0.1]),
       seed=st.integers(min_value=0, max_value=2**20))
def test_apply_A_is_symmetric_positive_definite(lens, lam, gap, seed):
    prob = synth.random_problem(len(lens), lens, 10, lam, seed, gap_frac=gap, hits_per_pix_min=4)
    nb = synth.to_numpy(prob)
    op = O.make_plan(nb["pix"], nb["psi"], nb["block_len"], nb["band"], nb["n_pix"])
    assume(op.n_obs > 0)   # not every pixel excised
    rng = np.random.default_rng(seed)
    u, v = rng.standard_normal((2, op.n_obs, 3))
    Au, Av = O.apply_A(op, u), O.apply_A(op, v)
    assert abs(np.vdot(u, Av) - np.vdot(Au, v)) <= 1e-11 * np.linalg.norm(u) * np.linalg.norm(Av)
    assert np.vdot(v, Av) > 0.0


@SETTINGS
@given(lens=st.lists(st.integers(min_value=0, max_value=400), min_size=1, max_size=3),
       n_poly=st.integers(min_value=0, max_value=4), n_az=st.integers(min_value=0, max_value=6),
       n_hwp=st.integers(min_value=0, max_value=3), interp=st.booleans(),
       seed=st.integers(min_value=0, max_value=2**20))
def test_template_filter_is_a_weighted_projection(lens, n_poly, n_az, n_hwp, interp, seed):
    assume(n_poly + n_az + 2 * n_hwp >= 1)
    n = sum(lens)
    assume(n > 0)
    rng = np.random.default_rng(seed)
    pix = rng.integers(0, 16, n).astype(np.int32)
    pix[rng.random(n) < 0.1] = -1                     # gaps
    psi = (rng.random(n) * 2 * np.pi).astype(np.float32)
    w = rng.uniform(0.5, 1.5, len(lens))
    op = O.make_plan(pix, psi, np.array(lens), w[:, None], 16)
    az = rng.uniform(0.0, 10.0, n).astype(np.float32)
    hwp = rng.uniform(0.0, 2 * np.pi, n).astype(np.float32)
    tm = O.Templates(n_poly=n_poly, n_az=n_az, n_hwp=n_hwp, interp=interp)
    t = rng.standard_normal(n)
    Ft = O.template_filter(op, w, tm, az, hwp, t)
    wb = np.repeat(w, lens)
    winv = np.where(op.lpix >= 0, 1.0 / wb, 0.0)
    FWF = O.template_filter(op, w, tm, az, hwp, winv * Ft)
    assert np.max(np.abs(FWF - Ft)) <= 1e-8 * max(1.0, np.max(np.abs(Ft)))
    assert np.all(Ft[op.lpix < 0] == 0.0)             # the filter carries the mask
