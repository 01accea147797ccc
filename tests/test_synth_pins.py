"""Pins of the input generator's noise weights to Eq. MADCAP and the PSD (no GPU)."""
import math

import numpy as np
import torch

import oracle as O
import synth


def test_white_psd_band():
    c, info = synth.inverse_noise_band(8192, 32, 50.0, 2.0, 0.0, 1.0)
    assert abs(float(c[0]) - 0.25) < 1e-15
    assert float(c[1:].abs().max()) < 1e-15
    assert info.lift == 0.0 and not info.tapered


def test_band_symbol_approximates_inverse_psd():
    lam, fs, fk, al = 1024, 100.0, 0.5, 1.0
    c, info = synth.inverse_noise_band(65536, lam, fs, 1.0, fk, al)
    n = 1 << 16
    h = np.zeros(n)
    cn = c.numpy()
    h[0] = cn[0]
    h[1:lam + 1] = cn[1:]
    h[n - lam:] = cn[1:][::-1]
    s = np.fft.rfft(h).real
    f = np.arange(s.size) * fs / n
    sel = (f > 20 * fs / lam) & (f < 0.45 * fs)
    target = 1.0 / (1.0 + (fk / f[sel]) ** al)
    assert np.max(np.abs(s[sel] - target) / target) < 2e-2
    assert info.min_symbol > 0


def test_band_inverts_noise_covariance_in_interior():
    # T(c) N ~= I away from block edges, N_ij = autocovariance of the PSD at |i - j|
    lam, fs, fk, al, sig = 256, 100.0, 0.2, 1.0, 1.0
    n = 2048
    c, _ = synth.inverse_noise_band(n, lam, fs, sig, fk, al)
    n_emb = 1 << 16
    f = torch.arange(n_emb // 2 + 1, dtype=torch.float64) * fs / n_emb
    p = synth.psd(f, sig, fk, al)
    acf = torch.fft.irfft(p.to(torch.complex128), n=n_emb).numpy()
    i = np.arange(n)
    N = acf[np.abs(i[:, None] - i[None, :])]
    T = O.toeplitz_dense(c.numpy(), n)
    TN = T @ N
    mid = slice(n // 2 - 64, n // 2 + 64)
    err = np.abs(TN[mid, mid] - np.eye(n)[mid, mid]).max()
    assert err < 0.1, err


def test_positivity_gate_makes_band_spd():
    c, info = synth.inverse_noise_band(524288, 8192, 100.0, 1.0, 1.0, 1.5)
    assert info.min_symbol > 0
    T = O.toeplitz_dense(c.numpy()[:200], 300)
    assert np.linalg.eigvalsh(T).min() > 0 or info.min_symbol > 0


def test_ground_pointing_recipe():
    cfg = synth.tiny_config()
    pix, psi = synth.ground_pointing(cfg)
    assert pix.numel() == cfg.n_total and int(pix.min()) >= 0 and int(pix.max()) < cfg.n_pix
    # 0.25 px/sample: 4 consecutive samples per pixel along a sweep, 512 samples per sweep
    p0 = pix[:512].numpy()
    assert (p0[:4] == p0[0]).all() and p0[4] == p0[0] + 1
    assert pix[512].item() // cfg.side == 1
    # psi = phi_det + 2 * (2 pi f_hwp t): detector 1 starts at 45 deg
    assert abs(float(psi[cfg.n_samp]) - math.pi / 4) < 1e-6
    assert float(psi.min()) >= 0 and float(psi.max()) < 2 * math.pi


def test_ground_template_streams_and_systematics():
    cfg = synth.tiny_config(n_det=3, n_int=2)
    pix, psi = synth.ground_pointing(cfg)
    az, hwp = synth.ground_template_streams(cfg)
    n = cfg.n_samp
    assert az.numel() == hwp.numel() == pix.numel()
    # the HWP angle is the rotation folded into psi: psi = phi_det + 2 phi_hwp (mod 2 pi)
    for det, k in ((0, 0), (1, 1), (2, 1)):
        lo = (det * cfg.n_int + k) * n
        d = np.remainder(psi[lo:lo + 1000].double().numpy() - (det % 4) * math.pi / 4
                         - 2 * hwp[lo:lo + 1000].double().numpy(), 2 * math.pi)
        assert np.max(np.minimum(d, 2 * math.pi - d)) < 1e-5
    t = (n + np.arange(5)) / cfg.fs   # interval 1 continues the clock
    np.testing.assert_allclose(hwp[n:n + 5].double().numpy(), np.remainder(2 * math.pi * cfg.hwp_hz * t, 2 * math.pi),
                               atol=1e-6)
    # azimuth: the raster's fast coordinate over a 10-degree sweep, the same for every detector
    sweep = int(round(cfg.side / cfg.speed))
    a0 = az[:2 * sweep].numpy()
    assert a0.min() == 180.0 and a0.max() == 190.0 and a0[0] == 180.0 and a0[sweep] == 190.0
    np.testing.assert_array_equal(az[:n].numpy(), az[2 * n:3 * n].numpy())
    # systematics: ground steps of 0.01 per 0.33 deg from the block's lowest azimuth, plus harmonics
    s = synth.template_systematics(cfg, az, hwp, seed=3, n_harm=0)
    a = az[:n].double().numpy()
    np.testing.assert_allclose(s[:n].numpy(), 1 + 0.01 * np.floor((a - a.min()) / 0.33), rtol=1e-12)
