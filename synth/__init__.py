"""Seeded synthetic inputs for the map-making problem (shared by the oracle tests and the CUDA path).

This module only *makes inputs*: scanning strategies (pixel index and polarisation angle per time
sample), a sky, 1/f noise realisations and the banded inverse-noise first rows that the map-maker
takes as its noise weights.  It implements none of the map-making arithmetic (no pointing
operator, no Toeplitz product, no preconditioner, no solver).

Everything is written with torch so the same recipe runs on the CPU (small parity cases, handed to
the oracle as numpy arrays) and on a CUDA device (full-size workloads, generated directly in HBM).

Recipe (stand-ins for the TOAST ground and satellite simulations of Sect. 4, which are not
available here):

* Ground raster: constant-elevation back-and-forth sweeps across a flat ``side x side`` patch at
  ``speed`` px/sample, one row advance per sweep, detectors offset on a focal-plane grid, a
  continuously rotating half-wave plate.  The stored angle is psi = phi_det + hwp_factor * phi_hwp so
  that the pointing weights (1, cos 2psi, sin 2psi) carry 2 phi + 4 phi_hwp as in the HWP data
  model of Sect. 2 (hwp_factor = 2).
* Satellite: spin + precession of a boresight on the sphere, equal-area pixels in (z, phi).
* Noise: stationary 1/f per (detector, interval) block with PSD sigma^2 (1 + (f_k/|f|)^alpha),
  P(0) := 0, drawn by circulant embedding.
* Weights: the first row of each inverse-noise Toeplitz block per Eq. MADCAP: inverse PSD on the
  circulant embedding grid, inverse FFT, cut at the half-bandwidth lambda (lambda + 1
  coefficients), with a positivity gate on the band's symbol.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict
from typing import Optional

import torch

SEED_BASE = 2112_03370_00


def seed_for(config_id: int, stream: int) -> int:
    """Seed of one random stream of one workload."""
    return SEED_BASE + 1000 * config_id + stream


# --------------------------------------------------------------------------------------------
# workload descriptions
# --------------------------------------------------------------------------------------------


@dataclass
class GroundConfig:
    """Raster-scan workload: n_det x n_int blocks of n_samp samples each (det-major)."""

    name: str = "tiny"
    config_id: int = 0
    n_det: int = 4
    n_int: int = 1
    n_samp: int = 65536
    side: int = 128
    speed: float = 0.25          # px per sample
    fs: float = 100.0            # Hz
    hwp_hz: float = 2.0
    hwp_factor: int = 2
    det_layout: str = "column"   # "column": offsets (0, j); "grid23": first n_det nodes of 23x23
    det_angle_mod: int = 4       # phi_j = (j mod det_angle_mod) * 45 deg
    cross_link: bool = False     # odd intervals sweep along y instead of x
    sigma_lo: float = 1.0
    sigma_hi: float = 1.0
    f_knee: float = 0.5
    alpha: float = 1.0
    lam: int = 1024
    tol: float = 1e-8
    sigma_I: float = 1.0
    sigma_QU: float = 0.1
    gap_frac: float = 0.0        # fraction of samples flagged (pix = -1), in short runs

    @property
    def n_blocks(self) -> int:
        return self.n_det * self.n_int

    @property
    def n_total(self) -> int:
        return self.n_blocks * self.n_samp

    @property
    def n_pix(self) -> int:
        return self.side * self.side


def tiny_config(**kw) -> GroundConfig:
    """4 dets x 65,536 samples at 100 Hz on a 128x128 patch, lambda = 1024, eps = 1e-8."""
    c = GroundConfig()
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def ground_config(**kw) -> GroundConfig:
    """512 dets x 4 intervals x 524,288 samples on a 1024x1024 patch, lambda = 8192."""
    c = GroundConfig(name="ground", config_id=1, n_det=512, n_int=4, n_samp=524288, side=1024,
                     speed=2.0, fs=100.0, hwp_hz=2.0, det_layout="grid23", det_angle_mod=4,
                     cross_link=True, sigma_lo=0.8, sigma_hi=1.2, f_knee=1.0, alpha=1.5,
                     lam=8192, tol=1e-6)
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def batched_config(**kw) -> GroundConfig:
    """Ground geometry cut to 128 dets x 1 interval x 524,288 samples."""
    c = ground_config(name="batched", config_id=3, n_det=128, n_int=1)
    for k, v in kw.items():
        setattr(c, k, v)
    return c


# --------------------------------------------------------------------------------------------
# scanning strategies
# --------------------------------------------------------------------------------------------


def _det_offsets(cfg: GroundConfig):
    j = torch.arange(cfg.n_det, dtype=torch.int64)
    if cfg.det_layout == "column":
        return torch.zeros_like(j), j
    if cfg.det_layout == "grid23":
        return (j % 23) - 11, (j // 23) - 11
    raise ValueError(cfg.det_layout)


def ground_pointing(cfg: GroundConfig, device="cpu", det_range: Optional[tuple] = None):
    """Pixel index (int32, -1 = flagged) and angle psi (float32, radians in [0, 2 pi)).

    Returns flat arrays over the blocks of detectors ``det_range`` (default: all), det-major,
    each block ``n_samp`` long.
    """
    d0, d1 = det_range if det_range is not None else (0, cfg.n_det)
    dev = torch.device(device)
    n = cfg.n_samp
    sweep = int(round(cfg.side / cfg.speed))
    i = torch.arange(n, device=dev, dtype=torch.int64)
    s = i // sweep
    u = torch.floor((i % sweep).to(torch.float64) * cfg.speed).to(torch.int64)
    xb = torch.where(s % 2 == 0, u, (cfg.side - 1) - u)
    yb = s % cfg.side
    dx_all, dy_all = _det_offsets(cfg)
    pix_out, psi_out = [], []
    two_pi = 2.0 * math.pi
    for det in range(d0, d1):
        dx, dy = int(dx_all[det]), int(dy_all[det])
        phi_det = (det % cfg.det_angle_mod) * (math.pi / 4.0)
        for k in range(cfg.n_int):
            if cfg.cross_link and (k % 2 == 1):
                px, py = yb, xb
            else:
                px, py = xb, yb
            px = (px + dx) % cfg.side
            py = (py + dy) % cfg.side
            pix = (py * cfg.side + px).to(torch.int32)
            t = (k * n + i).to(torch.float64) / cfg.fs
            ang = phi_det + cfg.hwp_factor * (two_pi * cfg.hwp_hz * t)
            psi = torch.remainder(ang, two_pi).to(torch.float32)
            psi = torch.where(psi >= two_pi, torch.zeros_like(psi), psi)   # f32 rounding up to 2 pi
            pix_out.append(pix)
            psi_out.append(psi)
    return torch.cat(pix_out), torch.cat(psi_out)


def flag_gaps(pix: torch.Tensor, frac: float, seed: int, run: int = 37) -> torch.Tensor:
    """Flag about ``frac`` of the samples as gaps (pix = -1) in runs of ``run`` samples."""
    if frac <= 0:
        return pix
    g = torch.Generator(device="cpu").manual_seed(seed)
    n_runs = max(1, int(frac * pix.numel() / run))
    starts = torch.randint(0, max(1, pix.numel() - run), (n_runs,), generator=g)
    idx = (starts[:, None] + torch.arange(run)[None, :]).reshape(-1).to(pix.device)
    out = pix.clone()
    out[idx] = -1
    return out


def ground_template_streams(cfg: GroundConfig, device="cpu", det_range: Optional[tuple] = None,
                            az_span_deg: float = 10.0):
    """Boresight azimuth and HWP angle per sample of the ground raster (det-major like
    ``ground_pointing``): float32 [N] each.

    The azimuth follows the raster's fast coordinate across a constant-elevation sweep of
    ``az_span_deg`` degrees (the same for every detector); the HWP angle is 2 pi hwp_hz t wrapped to
    [0, 2 pi), the rotation that ``ground_pointing`` folds into psi.
    """
    d0, d1 = det_range if det_range is not None else (0, cfg.n_det)
    dev = torch.device(device)
    n = cfg.n_samp
    sweep = int(round(cfg.side / cfg.speed))
    i = torch.arange(n, device=dev, dtype=torch.int64)
    s = i // sweep
    u = torch.floor((i % sweep).to(torch.float64) * cfg.speed)
    xb = torch.where(s % 2 == 0, u, (cfg.side - 1) - u)
    az_blk = (180.0 + az_span_deg * xb / (cfg.side - 1)).to(torch.float32)
    two_pi = 2.0 * math.pi
    hwp_int = []
    for k in range(cfg.n_int):
        t = (k * n + i).to(torch.float64) / cfg.fs
        h = torch.remainder(two_pi * cfg.hwp_hz * t, two_pi).to(torch.float32)
        hwp_int.append(torch.where(h >= two_pi, torch.zeros_like(h), h))
    hwp_det = torch.cat(hwp_int)
    n_det = d1 - d0
    return az_blk.repeat(n_det * cfg.n_int), hwp_det.repeat(n_det)


def template_systematics(cfg: GroundConfig, az: torch.Tensor, hwp: torch.Tensor, seed: int,
                         n_harm: int = 6, bin_deg: float = 0.33) -> torch.Tensor:
    """Ground pickup and HWP-synchronous signal per sample (float64 [N], det-major blocks of n_samp):

    * ground: a step function of azimuth, g_i = 1 + 0.01 i in bins of ``bin_deg`` from the
      sweep's lowest azimuth (the same ground map for every detector);
    * HWP: sum_n A_n (1 + eps t) cos(n phi) + B_n (1 + eps t) sin(n phi), n = 1..n_harm, with A_n,
      B_n ~ N(0.1, 0.001) per detector and a 1 % drift per 1000 s (t from the block's start).
    The shapes follow the template-marginalisation validation of Sect. 4 (Eqs. of the SSS and
    HWPSS signals); the amplitudes are in the sky's units.
    """
    n = cfg.n_samp
    nb = az.numel() // n
    dev = az.device
    a64 = az.to(torch.float64).view(nb, n)
    lo = a64.min(dim=1, keepdim=True).values
    g = 1.0 + 0.01 * torch.floor((a64 - lo) / bin_deg)
    gen = torch.Generator(device="cpu").manual_seed(seed)
    amp = (0.1 + 0.001 * torch.randn(cfg.n_det, 2, n_harm, generator=gen, dtype=torch.float64)).to(dev)
    t = torch.arange(n, dtype=torch.float64, device=dev) / cfg.fs
    drift = 1.0 + 0.01 * t / 1000.0
    out = g.reshape(-1).clone()
    phi = hwp.to(torch.float64).view(nb, n)
    for b in range(nb):
        det = b // cfg.n_int
        h = torch.zeros(n, dtype=torch.float64, device=dev)
        for m in range(1, n_harm + 1):
            h += amp[det, 0, m - 1] * torch.cos(m * phi[b]) + amp[det, 1, m - 1] * torch.sin(m * phi[b])
        out[b * n:(b + 1) * n] += drift * h
    return out


@dataclass
class SatelliteConfig:
    """Precessing spin scan on the full sky, equal-area lat-long pixels (rings in z x phi)."""

    name: str = "satellite"
    config_id: int = 2
    n_det: int = 64
    n_int: int = 1
    n_samp: int = 16777216
    fs: float = 20.0
    spin_period_s: float = 60.0
    prec_period_s: float = 96 * 60.0
    boresight_deg: float = 50.0
    spin_axis_deg: float = 45.0
    hwp_hz: float = 1.0
    hwp_factor: int = 2
    n_rings: int = 1536
    n_phi: int = 2048
    det_offset_deg: float = 0.5
    sigma_lo: float = 1.0
    sigma_hi: float = 1.0
    f_knee: float = 0.05
    alpha: float = 1.0
    lam: int = 4096
    tol: float = 1e-6
    sigma_I: float = 1.0
    sigma_QU: float = 0.1
    gap_frac: float = 0.0

    @property
    def n_blocks(self) -> int:
        return self.n_det * self.n_int

    @property
    def n_total(self) -> int:
        return self.n_blocks * self.n_samp

    @property
    def n_pix(self) -> int:
        return self.n_rings * self.n_phi


def satellite_config(**kw) -> SatelliteConfig:
    c = SatelliteConfig()
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def _rot_to(axis: torch.Tensor, v: torch.Tensor) -> torch.Tensor:
    """Rotate vectors v given in a frame whose z axis is ``axis`` (both [n, 3]) to the sky frame."""
    z = axis / axis.norm(dim=1, keepdim=True)
    ref = torch.zeros_like(z)
    ref[:, 0] = 1.0
    alt = torch.zeros_like(z)
    alt[:, 1] = 1.0
    use_alt = (z[:, 0].abs() > 0.9)[:, None]
    ref = torch.where(use_alt, alt, ref)
    x = torch.linalg.cross(ref, z)
    x = x / x.norm(dim=1, keepdim=True)
    y = torch.linalg.cross(z, x)
    return v[:, :1] * x + v[:, 1:2] * y + v[:, 2:3] * z


def satellite_pointing(cfg: SatelliteConfig, device="cpu", det_range: Optional[tuple] = None):
    """Pixel (int32) and angle (float32) of a precessing spin scan with a continuously rotating
    half-wave plate: the anti-sun axis turns once over the run, the spin axis precesses about it
    at spin_axis_deg, the boresight spins at boresight_deg about the spin axis.  Detector j sits
    on a small focal-plane grid (offsets up to det_offset_deg) at angle (j mod 4) * 45 deg."""
    d0, d1 = det_range if det_range is not None else (0, cfg.n_det)
    dev = torch.device(device)
    n = cfg.n_samp
    t = torch.arange(n, dtype=torch.float64, device=dev) / cfg.fs
    two_pi = 2.0 * math.pi
    T = n / cfg.fs
    lon = two_pi * t / T
    sun = torch.stack([torch.cos(lon), torch.sin(lon), torch.zeros_like(lon)], dim=1)
    a = math.radians(cfg.spin_axis_deg)
    wp = two_pi * t / cfg.prec_period_s
    spin_local = torch.stack([math.sin(a) * torch.cos(wp), math.sin(a) * torch.sin(wp),
                              torch.full_like(wp, math.cos(a))], dim=1)
    spin = _rot_to(sun, spin_local)
    bang = math.radians(cfg.boresight_deg)
    ws = two_pi * t / cfg.spin_period_s
    b_local = torch.stack([math.sin(bang) * torch.cos(ws), math.sin(bang) * torch.sin(ws),
                           torch.full_like(ws, math.cos(bang))], dim=1)
    bore = _rot_to(spin, b_local)
    # scan direction (boresight velocity) gives the focal-plane orientation
    v_local = torch.stack([-torch.sin(ws), torch.cos(ws), torch.zeros_like(ws)], dim=1)
    vel = _rot_to(spin, v_local)
    vel = vel - (vel * bore).sum(1, keepdim=True) * bore
    vel = vel / vel.norm(dim=1, keepdim=True)
    crs = torch.linalg.cross(bore, vel)
    g = int(math.ceil(math.sqrt(max(cfg.n_det, 1))))
    pix_out, psi_out = [], []
    for det in range(d0, d1):
        ox = ((det % g) / max(g - 1, 1) - 0.5) * 2 * math.radians(cfg.det_offset_deg)
        oy = ((det // g) / max(g - 1, 1) - 0.5) * 2 * math.radians(cfg.det_offset_deg)
        p = bore + ox * vel + oy * crs
        p = p / p.norm(dim=1, keepdim=True)
        z = p[:, 2].clamp(-1.0, 1.0)
        phi = torch.remainder(torch.atan2(p[:, 1], p[:, 0]), two_pi)
        ring = torch.clamp(torch.floor((z + 1.0) * 0.5 * cfg.n_rings), 0, cfg.n_rings - 1).long()
        col = torch.clamp(torch.floor(phi / two_pi * cfg.n_phi), 0, cfg.n_phi - 1).long()
        pix = (ring * cfg.n_phi + col).to(torch.int32)
        # polarisation angle: detector angle + orientation of the scan w.r.t. the meridian + HWP
        east = torch.stack([-torch.sin(phi), torch.cos(phi), torch.zeros_like(phi)], dim=1)
        north = torch.linalg.cross(p, east)
        orient = torch.atan2((vel * east).sum(1), (vel * north).sum(1))
        ang = (det % 4) * (math.pi / 4.0) + orient + cfg.hwp_factor * (two_pi * cfg.hwp_hz * t)
        psi = torch.remainder(ang, two_pi).to(torch.float32)
        psi = torch.where(psi >= two_pi, torch.zeros_like(psi), psi)
        pix_out.append(pix)
        psi_out.append(psi)
    return torch.cat(pix_out), torch.cat(psi_out)


def make_satellite_problem(cfg: SatelliteConfig, device="cpu", det_range: Optional[tuple] = None,
                           with_noise: bool = True) -> "Problem":
    """Satellite-like problem: pointing, bands (shared shape, per-detector scale), sky and data."""
    d0, d1 = det_range if det_range is not None else (0, cfg.n_det)
    dev = torch.device(device)
    n_det = d1 - d0
    pix = torch.empty(n_det * cfg.n_samp, dtype=torch.int32, device=dev)
    psi = torch.empty(n_det * cfg.n_samp, dtype=torch.float32, device=dev)
    for j in range(d0, d1):   # one detector at a time keeps the float64 temporaries small
        pj, sj = satellite_pointing(cfg, device=dev, det_range=(j, j + 1))
        pix[(j - d0) * cfg.n_samp:(j - d0 + 1) * cfg.n_samp] = pj
        psi[(j - d0) * cfg.n_samp:(j - d0 + 1) * cfg.n_samp] = sj
    gs = torch.Generator(device="cpu").manual_seed(seed_for(cfg.config_id, 2))
    sig_all = cfg.sigma_lo + (cfg.sigma_hi - cfg.sigma_lo) * torch.rand(
        cfg.n_det, generator=gs, dtype=torch.float64)
    sig = sig_all[d0:d1]
    shape, info = inverse_noise_band(cfg.n_samp, cfg.lam, cfg.fs, 1.0, cfg.f_knee, cfg.alpha)
    band = torch.stack([shape / (sig[j] ** 2) for j in range(n_det)])
    m = sky(cfg.n_pix, cfg.sigma_I, cfg.sigma_QU, seed_for(cfg.config_id, 1), device=dev)
    dd = torch.zeros(pix.numel(), dtype=torch.float64, device=dev)
    gn = torch.Generator(device=dev).manual_seed(seed_for(cfg.config_id, 100) + 7919 * d0)
    for j in range(n_det):
        lo, hi = j * cfg.n_samp, (j + 1) * cfg.n_samp
        pl = pix[lo:hi].long()
        two = 2.0 * psi[lo:hi].to(torch.float64)
        dd[lo:hi] = m[pl, 0] + torch.cos(two) * m[pl, 1] + torch.sin(two) * m[pl, 2]
        if with_noise:
            dd[lo:hi] += noise_block(cfg.n_samp, cfg.fs, float(sig[j]), cfg.f_knee, cfg.alpha, gn, dev)
    block_len = torch.full((n_det,), cfg.n_samp, dtype=torch.int64)
    return Problem(n_det=n_det, n_int=1, block_len=block_len, n_pix=cfg.n_pix, pix=pix, psi=psi,
                   lam=cfg.lam, band=band, d=dd, m_sky=m, tol=cfg.tol, band_info=info, sigmas=sig)


# --------------------------------------------------------------------------------------------
# sky, noise, weights
# --------------------------------------------------------------------------------------------


def sky(n_pix: int, sigma_I: float, sigma_QU: float, seed: int, device="cpu") -> torch.Tensor:
    """I ~ N(0, sigma_I^2), Q, U ~ N(0, sigma_QU^2), i.i.d. per pixel: float64 [n_pix, 3]."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    m = torch.randn(n_pix, 3, generator=g, dtype=torch.float64)
    m[:, 0] *= sigma_I
    m[:, 1:] *= sigma_QU
    return m.to(device)


def psd(f: torch.Tensor, sigma: float, f_knee: float, alpha: float) -> torch.Tensor:
    """sigma^2 (1 + (f_knee/|f|)^alpha), per-sample variance density; P(0) := 0 (1/f limit)."""
    af = f.abs()
    out = torch.zeros_like(af)
    nz = af > 0
    if f_knee > 0:
        out[nz] = sigma * sigma * (1.0 + (f_knee / af[nz]) ** alpha)
    else:
        out[nz] = sigma * sigma
        out[~nz] = sigma * sigma
    return out


def noise_block(n: int, fs: float, sigma: float, f_knee: float, alpha: float,
                gen: torch.Generator, device="cpu") -> torch.Tensor:
    """One stationary noise stream of length n by circulant embedding on 2^ceil(log2 2n) points."""
    n_emb = 1 << int(math.ceil(math.log2(2 * n)))
    w = torch.randn(n_emb, generator=gen, dtype=torch.float64, device=gen.device).to(device)
    W = torch.fft.rfft(w)
    f = torch.arange(W.numel(), dtype=torch.float64, device=device) * (fs / n_emb)
    W = W * torch.sqrt(psd(f, sigma, f_knee, alpha))
    return torch.fft.irfft(W, n=n_emb)[:n]


def symbol_min(c: torch.Tensor) -> float:
    """Minimum over a fine grid of s(w) = c0 + 2 sum_k c_k cos(k w) (band's Fourier symbol)."""
    lam = c.numel() - 1
    n_s = 1 << int(math.ceil(math.log2(16 * (lam + 1))))
    h = torch.zeros(n_s, dtype=torch.float64)
    h[0] = c[0]
    if lam > 0:
        h[1:lam + 1] = c[1:]
        h[n_s - lam:] = torch.flip(c[1:], [0])
    return float(torch.fft.rfft(h).real.min())


@dataclass
class BandInfo:
    tapered: bool = False
    lift: float = 0.0
    min_symbol: float = 0.0


def inverse_noise_band(n_block: int, lam: int, fs: float, sigma: float, f_knee: float,
                       alpha: float, gauss_taper: bool = False):
    """First row c[0..lam] of the approximate inverse-noise Toeplitz block (Eq. MADCAP).

    The inverse PSD is sampled on the circulant-embedding grid of n_fft = 2^ceil(log2 max(n_block,
    4(lam+1))) points (1/P(0) := 0), inverse-transformed and cut at |tau| <= lam.  If the cut band
    has a non-positive symbol it is tapered by a Gaussian window of width lam/2 (the smoothing of
    Sect. 3.2) and, if still needed, lifted on the diagonal so every finite block is SPD.
    """
    n_fft = 1 << int(math.ceil(math.log2(max(n_block, 4 * (lam + 1)))))
    f = torch.arange(n_fft // 2 + 1, dtype=torch.float64) * (fs / n_fft)
    p = psd(f, sigma, f_knee, alpha)
    inv = torch.zeros_like(p)
    nz = p > 0
    inv[nz] = 1.0 / p[nz]
    c = torch.fft.irfft(inv.to(torch.complex128), n=n_fft)[: lam + 1].clone()
    info = BandInfo()
    if gauss_taper and lam > 0:
        tau = torch.arange(lam + 1, dtype=torch.float64)
        c = c * torch.exp(-0.5 * (tau / (lam / 2.0)) ** 2)
        info.tapered = True
    smin = symbol_min(c)
    if smin <= 0 and not info.tapered and lam > 0:
        tau = torch.arange(lam + 1, dtype=torch.float64)
        c = c * torch.exp(-0.5 * (tau / (lam / 2.0)) ** 2)
        info.tapered = True
        smin = symbol_min(c)
    if smin <= 0:
        lift = abs(smin) * (1.0 + 1e-3) + 1e-12 * float(c[0])
        c[0] += lift
        info.lift = lift
        smin = symbol_min(c)
    info.min_symbol = smin
    return c, info


# --------------------------------------------------------------------------------------------
# assembled problems
# --------------------------------------------------------------------------------------------


@dataclass
class Problem:
    """One map-making problem: all arrays are torch tensors on one device."""

    n_det: int
    n_int: int
    block_len: torch.Tensor      # int64 [n_blocks] (host)
    n_pix: int
    pix: torch.Tensor            # int32 [N], -1 = gap
    psi: torch.Tensor            # float32 [N]
    lam: int
    band: torch.Tensor           # float64 [n_blocks, lam + 1]
    d: Optional[torch.Tensor]    # float64 [N] (or None)
    m_sky: Optional[torch.Tensor]
    tol: float
    band_info: BandInfo = field(default_factory=BandInfo)
    sigmas: Optional[torch.Tensor] = None

    @property
    def n_total(self) -> int:
        return int(self.pix.numel())


def make_ground_problem(cfg: GroundConfig, device="cpu", with_noise: bool = True,
                        with_signal: bool = True, det_range: Optional[tuple] = None,
                        n_real: int = 1, real_offset: int = 0) -> Problem:
    """Build one ground-raster problem (pointing, bands, sky, data) for ``cfg``.

    ``det_range`` restricts to a contiguous subset of detectors (same per-detector recipe and
    seeds as the full problem).  ``n_real`` > 1 returns d as [n_real, N] noise realisations
    (realisation r uses noise stream 100 + r + real_offset).
    """
    d0, d1 = det_range if det_range is not None else (0, cfg.n_det)
    dev = torch.device(device)
    pix, psi = ground_pointing(cfg, device=dev, det_range=(d0, d1))
    if cfg.gap_frac > 0:
        pix = flag_gaps(pix.cpu(), cfg.gap_frac, seed_for(cfg.config_id, 7)).to(dev)
    n_det = d1 - d0
    gs = torch.Generator(device="cpu").manual_seed(seed_for(cfg.config_id, 2))
    sig_all = cfg.sigma_lo + (cfg.sigma_hi - cfg.sigma_lo) * torch.rand(
        cfg.n_det, generator=gs, dtype=torch.float64)
    sig = sig_all[d0:d1]
    shape, info = inverse_noise_band(cfg.n_samp, cfg.lam, cfg.fs, 1.0, cfg.f_knee, cfg.alpha)
    band = torch.empty(n_det * cfg.n_int, cfg.lam + 1, dtype=torch.float64)
    for j in range(n_det):
        band[j * cfg.n_int:(j + 1) * cfg.n_int] = shape / (sig[j] ** 2)
    block_len = torch.full((n_det * cfg.n_int,), cfg.n_samp, dtype=torch.int64)
    m = sky(cfg.n_pix, cfg.sigma_I, cfg.sigma_QU, seed_for(cfg.config_id, 1), device=dev)
    d = None
    if with_noise or with_signal:
        reals = []
        for r in range(n_real):
            dd = torch.zeros(pix.numel(), dtype=torch.float64, device=dev)
            gn = None
            if with_noise:
                stream = 100 + r + real_offset
                gn = torch.Generator(device=dev).manual_seed(seed_for(cfg.config_id, stream)
                                                             + 7919 * d0)
            for j in range(n_det):
                for k in range(cfg.n_int):
                    lo = (j * cfg.n_int + k) * cfg.n_samp
                    hi = lo + cfg.n_samp
                    if with_signal:
                        pb = pix[lo:hi]
                        pl = pb.clamp(min=0).long()
                        two = 2.0 * psi[lo:hi].to(torch.float64)
                        sig_t = m[pl, 0] + torch.cos(two) * m[pl, 1] + torch.sin(two) * m[pl, 2]
                        dd[lo:hi] += torch.where(pb >= 0, sig_t, torch.zeros_like(sig_t))
                    if with_noise:
                        dd[lo:hi] += noise_block(cfg.n_samp, cfg.fs, float(sig[j]), cfg.f_knee,
                                                 cfg.alpha, gn, dev)
            reals.append(dd)
        d = reals[0] if n_real == 1 else torch.stack(reals)
    return Problem(n_det=n_det, n_int=cfg.n_int, block_len=block_len, n_pix=cfg.n_pix, pix=pix,
                   psi=psi, lam=cfg.lam, band=band, d=d, m_sky=m, tol=cfg.tol, band_info=info,
                   sigmas=sig)


def random_problem(n_blocks: int, block_len, n_pix: int, lam: int, seed: int,
                   gap_frac: float = 0.0, f_knee: float = 0.5, alpha: float = 1.0,
                   hits_per_pix_min: int = 0, device="cpu") -> Problem:
    """Small unstructured problem: random pixels and angles, arbitrary (ragged) block lengths.

    Used for edge cases (ragged blocks, blocks shorter than lambda, gaps, lambda = 0).  Angles are
    uniform, so every pixel with a few hits is well conditioned.
    """
    g = torch.Generator(device="cpu").manual_seed(seed)
    if isinstance(block_len, int):
        block_len = [block_len] * n_blocks
    bl = torch.tensor(block_len, dtype=torch.int64)
    n = int(bl.sum())
    pix = torch.randint(0, n_pix, (n,), generator=g, dtype=torch.int64)
    if hits_per_pix_min > 0:
        base = torch.arange(n_pix).repeat_interleave(hits_per_pix_min)
        k = min(base.numel(), n)
        perm = torch.randperm(n, generator=g)[:k]
        pix[perm] = base[:k]
    pix = pix.to(torch.int32)
    psi = (torch.rand(n, generator=g, dtype=torch.float64) * 2 * math.pi).to(torch.float32)
    if gap_frac > 0:
        gm = torch.rand(n, generator=g) < gap_frac
        pix[gm] = -1
    band = torch.empty(n_blocks, lam + 1, dtype=torch.float64)
    for b in range(n_blocks):
        sig = 0.8 + 0.4 * float(torch.rand(1, generator=g))
        shape, _ = inverse_noise_band(max(int(bl[b]), 1), lam, 100.0, 1.0, f_knee, alpha)
        band[b] = shape / sig ** 2
    m = sky(n_pix, 1.0, 0.1, seed + 1)
    two = 2.0 * psi.to(torch.float64)
    pl = pix.clamp(min=0).long()
    d = torch.where(pix >= 0, m[pl, 0] + torch.cos(two) * m[pl, 1] + torch.sin(two) * m[pl, 2],
                    torch.zeros(n, dtype=torch.float64))
    d = d + 0.1 * torch.randn(n, generator=g, dtype=torch.float64)
    return Problem(n_det=n_blocks, n_int=1, block_len=bl, n_pix=n_pix, pix=pix.to(device),
                   psi=psi.to(device), lam=lam, band=band, d=d.to(device), m_sky=m, tol=1e-8)


def to_numpy(prob: Problem) -> dict:
    """The problem as plain numpy arrays (what the oracle consumes)."""
    out = dict(n_det=prob.n_det, n_int=prob.n_int, n_pix=prob.n_pix, lam=prob.lam, tol=prob.tol,
               block_len=prob.block_len.cpu().numpy(), pix=prob.pix.cpu().numpy(),
               psi=prob.psi.cpu().numpy(), band=prob.band.cpu().numpy())
    if prob.d is not None:
        out["d"] = prob.d.cpu().numpy()
    if prob.m_sky is not None:
        out["m_sky"] = prob.m_sky.cpu().numpy()
    return out
