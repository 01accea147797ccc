"""Plain FP64 CPU oracle of maximum-likelihood map-making (El Bouhargani et al., MAPPRAISER).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  It shares no code, tables or helpers with the CUDA library
and must never be used as a fallback for it.

Every function follows a passage of the paper (Sect. = section, Eq. = equation, Algorithm = the
numbered algorithm) and is written for a reader to check by eye: numpy/scipy in float64, no blocking
or fusion beyond what the definition states.

Notation (Sect. 2 and 3):
  N samples t; block b = (detector, stationary interval), blocks stored contiguously, det-major.
  pix[t]  global pixel (-1 = flagged sample), psi[t] polarisation angle (float32 on input).
  Pointing row of sample t: weights w_t = (1, cos 2psi_t, sin 2psi_t) at pixel p_t (Eq. of the HWP
  data model, with 2psi = 2phi + 4phi_hwp).
  N^-1 = blockdiag_b T(c_b), T(c)_ij = c_|i-j| for |i-j| <= lambda inside block b, else 0
  (Eq. MADCAP; lambda + 1 coefficients c_0..c_lambda; no wrap, no coupling across blocks).
  G zeroes flagged samples and samples of excised pixels on both sides of N^-1 (gstbmm, Sect. 3.1).
  A = P~^T N^-1 P~, b = P~^T N^-1 G d, with P~ = G P restricted to the n_obs kept pixels.
  M_BD = (P~^T diag(N^-1) P~)^-1, a 3x3 block per pixel (Sect. 3.2, block-Jacobi).

Parity pins live in tests/test_oracle_pins.py.  Functions without a pin: none (the 2lvl
construction is pinned by (I - AQ)AZ = 0 and M_2lvl A Z = Z; block CG by s = 1 == PCG; enlarged
CG by t = 1 == PCG iterate by iterate, the dense solve for t = 2..8 in both variants, the
Galerkin condition P_k^T R_k = 0, and Orthomin == Orthodir on a well-conditioned problem; the
a-priori deflation space by hit counts taken sample by sample, the partition of unity, and the
same deflation identities as the a-posteriori one; the noise-weight estimator by one-sided
Parseval, a pure cosine, gap handling by hand, exact recovery of a noise-free model, a noise
realisation with known parameters, and the closed form and a brute-force inverse DFT of the band;
the template filter by F_T T = 0, symmetry and positivity, closed forms of every template column,
the no-template limit equal to the diagonal-weighted operator, and exact recovery of a map from
data that carries template signals).
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field
from typing import Optional

import numpy as np
import scipy.linalg
import scipy.optimize
import scipy.signal
import scipy.special

__all__ = [
    "pointing_weights", "block_offsets", "sample_block", "bd_blocks", "excise", "OraclePlan",
    "make_plan", "unpoint", "point", "toeplitz_direct", "toeplitz_fft", "toeplitz_dense",
    "apply_A", "rhs", "precond_bd", "pcg", "PCGResult", "dense_A", "dense_solve",
    "block_cg", "lanczos", "TwoLevel", "two_level_from_lanczos", "binned_map",
]


# ------------------------------------------------------------------------------------------
# pointing (Sect. 2, data model with a half-wave plate; Sect. 3.1 MAPMAT un-pointing/pointing)
# ------------------------------------------------------------------------------------------


def pointing_weights(psi) -> np.ndarray:
    """Row weights (1, cos 2psi, sin 2psi) of the pointing matrix, float64 [N, 3].

    HWP data model of Sect. 2: d_t = I + cos(2phi + 4phi_hwp) Q + sin(...) U.  The stored angle is
    psi with 2psi = 2phi + 4phi_hwp; the float32 input angle is promoted to float64 first.
    """
    two = 2.0 * np.asarray(psi, dtype=np.float64)
    w = np.empty((two.size, 3), dtype=np.float64)
    w[:, 0] = 1.0
    w[:, 1] = np.cos(two)
    w[:, 2] = np.sin(two)
    return w


def block_offsets(block_len) -> np.ndarray:
    """Start offsets of the contiguous (detector, interval) blocks, length n_blocks + 1."""
    bl = np.asarray(block_len, dtype=np.int64)
    return np.concatenate([[0], np.cumsum(bl)])


def sample_block(block_len) -> np.ndarray:
    """Block index of every sample."""
    bl = np.asarray(block_len, dtype=np.int64)
    return np.repeat(np.arange(bl.size), bl)


# ------------------------------------------------------------------------------------------
# block-Jacobi blocks and pixel excision (Sect. 2.4 degeneracies; Sect. 3.2 preconditioners)
# ------------------------------------------------------------------------------------------


def bd_blocks(pix, psi, block_len, band, n_pix):
    """Per global pixel: B_p = sum_{t: p_t = p} c_0,b(t) w_t w_t^T (3x3) and the hit count.

    Block-Jacobi preconditioner of Sect. 3.2: P^T diag(N^-1) P, with diag(N^-1) on sample t equal
    to the first coefficient c_0 of its block.
    """
    pix = np.asarray(pix)
    ok = pix >= 0
    w = pointing_weights(psi)
    c0 = np.asarray(band, dtype=np.float64)[:, 0][sample_block(block_len)]
    p = pix[ok].astype(np.int64)
    wk = w[ok]
    ck = c0[ok]
    B = np.zeros((n_pix, 3, 3), dtype=np.float64)
    for i in range(3):
        for j in range(3):
            B[:, i, j] = np.bincount(p, weights=ck * wk[:, i] * wk[:, j], minlength=n_pix)
    hits = np.bincount(p, minlength=n_pix).astype(np.int64)
    return B, hits


def excise(B, hits, cond_max: float = 1e3):
    """Keep mask and condition numbers (Sect. 2.4: threshold on the cond of each 3x3 block).

    A pixel is kept when it has >= 3 hits and cond_2(B_p) = lambda_max / lambda_min <= cond_max
    (ties kept).  The paper gives no threshold value; 1e3 is the default reading.
    """
    ev = np.linalg.eigvalsh(B)
    lo, hi = ev[:, 0], ev[:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        cond = np.where(lo > 0, hi / np.where(lo > 0, lo, 1.0), np.inf)
    keep = (hits >= 3) & (cond <= cond_max)
    return keep, cond


@dataclass
class OraclePlan:
    """Everything the oracle needs about one problem after pixel compaction."""

    block_len: np.ndarray
    offsets: np.ndarray
    band: np.ndarray             # [n_blocks, lambda + 1]
    lam: int
    n_pix: int
    pix: np.ndarray              # global pixel per sample
    lpix: np.ndarray             # local (compacted) pixel per sample, -1 = masked (G)
    w: np.ndarray                # [N, 3]
    keep: np.ndarray             # [n_pix] bool
    obs_to_global: np.ndarray    # [n_obs]
    B: np.ndarray                # [n_obs, 3, 3] BD blocks of kept pixels
    Minv: np.ndarray             # [n_obs, 3, 3]
    cond: np.ndarray             # [n_pix]
    hits: np.ndarray             # [n_pix]
    toeplitz: str = "fft"

    @property
    def n_obs(self) -> int:
        return int(self.obs_to_global.size)

    @property
    def mask(self) -> np.ndarray:
        return self.lpix >= 0


def make_plan(pix, psi, block_len, band, n_pix, cond_max: float = 1e3,
              toeplitz: str = "fft") -> OraclePlan:
    """Pixel compaction (Sect. 3.1: local indexation of observed pixels) plus BD + excision.

    Local ids follow ascending global pixel order over the kept pixels.
    """
    pix = np.asarray(pix, dtype=np.int64)
    band = np.asarray(band, dtype=np.float64)
    B, hits = bd_blocks(pix, psi, block_len, band, n_pix)
    keep, cond = excise(B, hits, cond_max)
    obs = np.nonzero(keep)[0]
    lid = -np.ones(n_pix, dtype=np.int64)
    lid[obs] = np.arange(obs.size)
    lpix = np.where(pix >= 0, lid[np.clip(pix, 0, None)], -1)
    Bk = B[obs]
    Minv = np.linalg.inv(Bk) if obs.size else np.zeros((0, 3, 3))
    return OraclePlan(block_len=np.asarray(block_len, dtype=np.int64),
                      offsets=block_offsets(block_len), band=band, lam=band.shape[1] - 1,
                      n_pix=n_pix, pix=pix, lpix=lpix, w=pointing_weights(psi), keep=keep,
                      obs_to_global=obs, B=Bk, Minv=Minv, cond=cond, hits=hits,
                      toeplitz=toeplitz)


def unpoint(plan: OraclePlan, m) -> np.ndarray:
    """t = P~ m (Sect. 3.1 un-pointing): t_i = sum_j w_ij m[p_i, j]; 0 for masked samples."""
    m = np.asarray(m, dtype=np.float64).reshape(-1, 3)
    ok = plan.lpix >= 0
    t = np.zeros(plan.lpix.size, dtype=np.float64)
    p = plan.lpix[ok]
    t[ok] = (plan.w[ok] * m[p]).sum(axis=1)
    return t


def point(plan: OraclePlan, y) -> np.ndarray:
    """m = P~^T y (Sect. 3.1 pointing): m[p, j] = sum_{t: p_t = p} w_tj y_t over unmasked t."""
    y = np.asarray(y, dtype=np.float64)
    ok = plan.lpix >= 0
    p = plan.lpix[ok]
    out = np.empty((plan.n_obs, 3), dtype=np.float64)
    for j in range(3):
        out[:, j] = np.bincount(p, weights=plan.w[ok, j] * y[ok], minlength=plan.n_obs)
    return out


# ------------------------------------------------------------------------------------------
# N^-1: symmetric banded Toeplitz blocks (Eq. MADCAP; Sect. 3.1 stbmm / gstbmm)
# ------------------------------------------------------------------------------------------


def toeplitz_direct(band, block_len, t) -> np.ndarray:
    """y = blockdiag_b T(c_b) t by the definition: y_i = sum_{|i-j|<=lambda, j in block} c_|i-j| t_j."""
    band = np.asarray(band, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    off = block_offsets(block_len)
    lam = band.shape[1] - 1
    y = np.zeros_like(t)
    for b in range(band.shape[0]):
        lo, hi = off[b], off[b + 1]
        tb = t[lo:hi]
        n = tb.size
        yb = band[b, 0] * tb.copy()
        for k in range(1, min(lam, n - 1) + 1):
            yb[:-k] += band[b, k] * tb[k:]
            yb[k:] += band[b, k] * tb[:-k]
        y[lo:hi] = yb
    return y


def toeplitz_fft(band, block_len, t) -> np.ndarray:
    """Same product as :func:`toeplitz_direct` computed as a linear convolution per block.

    Each block's output is the centred part of the full convolution of the block with the
    symmetric kernel (c_lam, ..., c_1, c_0, c_1, ..., c_lam) (library FFT convolution), which is the
    banded Toeplitz product with no wrap-around and no coupling across blocks.
    """
    band = np.asarray(band, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    off = block_offsets(block_len)
    lam = band.shape[1] - 1
    y = np.zeros_like(t)
    for b in range(band.shape[0]):
        lo, hi = off[b], off[b + 1]
        if hi == lo:
            continue
        h = np.concatenate([band[b, :0:-1], band[b]])
        full = scipy.signal.fftconvolve(t[lo:hi], h, mode="full")
        y[lo:hi] = full[lam:lam + (hi - lo)]
    return y


def toeplitz_dense(c, n) -> np.ndarray:
    """Dense n x n banded Toeplitz T(c) (tiny sizes only)."""
    c = np.asarray(c, dtype=np.float64)
    lam = c.size - 1
    i = np.arange(n)
    k = np.abs(i[:, None] - i[None, :])
    T = np.zeros((n, n), dtype=np.float64)
    inb = k <= lam
    T[inb] = c[k[inb]]
    return T


def _toeplitz(plan: OraclePlan, t):
    if plan.toeplitz == "direct":
        return toeplitz_direct(plan.band, plan.block_len, t)
    return toeplitz_fft(plan.band, plan.block_len, t)


# ------------------------------------------------------------------------------------------
# system matrix, right-hand side, preconditioner (Sect. 3.2)
# ------------------------------------------------------------------------------------------


def apply_A(plan: OraclePlan, x) -> np.ndarray:
    """A x = P~^T N^-1 P~ x, right to left: un-point, block-Toeplitz product, point (Sect. 3.2)."""
    return point(plan, _toeplitz(plan, unpoint(plan, x)))


def rhs(plan: OraclePlan, d) -> np.ndarray:
    """b = P~^T N^-1 G d (the estimator of Sect. 2 with F_T = W^-1 = N^-1; G on both sides)."""
    gd = np.where(plan.lpix >= 0, np.asarray(d, dtype=np.float64), 0.0)
    return point(plan, _toeplitz(plan, gd))


def precond_bd(plan: OraclePlan, r) -> np.ndarray:
    """z = M_BD r with M_BD = (P~^T diag(N^-1) P~)^-1, one 3x3 block per kept pixel."""
    r = np.asarray(r, dtype=np.float64).reshape(-1, 3)
    return np.einsum("pij,pj->pi", plan.Minv, r)


def binned_map(plan: OraclePlan, d) -> np.ndarray:
    """M_BD P~^T diag(N^-1) G d: the map of the diagonal-weights (lambda = 0) special case."""
    c0 = plan.band[:, 0][sample_block(plan.block_len)]
    gd = np.where(plan.lpix >= 0, np.asarray(d, dtype=np.float64), 0.0)
    return precond_bd(plan, point(plan, c0 * gd))


# ------------------------------------------------------------------------------------------
# Algorithm 1: PCG
# ------------------------------------------------------------------------------------------


@dataclass
class PCGResult:
    x: np.ndarray
    iters: int
    converged: bool
    rel_res: float                      # recursive ||r|| / ||b||
    history: list = field(default_factory=list)
    iterates: Optional[list] = None


def pcg(plan: OraclePlan, b, tol: float = 1e-6, max_iter: int = 10000, precond=None,
        keep_iterates: bool = False, apply=None) -> PCGResult:
    """Algorithm 1 (PCG) with x_0 = 0 and the stopping rule ||r_{k+1}||_2 < eps ||b||_2.

    The residual is the recursive one of the algorithm (unpreconditioned 2-norm over all IQU
    unknowns).  ``precond`` defaults to M_BD; ``apply`` defaults to A.  ``iters`` counts the
    A-applications performed inside the loop (x_0 = 0, so r_0 = b needs none).
    """
    A = apply if apply is not None else (lambda v: apply_A(plan, v))
    M = precond if precond is not None else (lambda v: precond_bd(plan, v))
    b = np.asarray(b, dtype=np.float64).reshape(-1, 3)
    x = np.zeros_like(b)
    r = b.copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return PCGResult(x=x, iters=0, converged=True, rel_res=0.0)
    z = M(r)
    p = z.copy()
    rz = float(np.vdot(r, z))
    hist = []
    its = [] if keep_iterates else None
    k = 0
    converged = False
    rel = 1.0
    while k < max_iter:
        Ap = A(p)
        alpha = rz / float(np.vdot(Ap, p))
        x = x + alpha * p
        r = r - alpha * Ap
        k += 1
        rel = float(np.linalg.norm(r)) / bnorm
        hist.append(rel)
        if keep_iterates:
            its.append(x.copy())
        if rel < tol:
            converged = True
            break
        z = M(r)
        rz_new = float(np.vdot(r, z))
        beta = rz_new / rz
        rz = rz_new
        p = z + beta * p
    return PCGResult(x=x, iters=k, converged=converged, rel_res=rel, history=hist, iterates=its)


# ------------------------------------------------------------------------------------------
# dense references for tiny problems
# ------------------------------------------------------------------------------------------


def dense_A(plan: OraclePlan) -> np.ndarray:
    """A = P~^T N^-1 P~ assembled densely from a dense P~ and dense T(c_b) blocks (tiny only)."""
    n = plan.lpix.size
    Pd = np.zeros((n, 3 * plan.n_obs), dtype=np.float64)
    ok = np.nonzero(plan.lpix >= 0)[0]
    for j in range(3):
        Pd[ok, 3 * plan.lpix[ok] + j] = plan.w[ok, j]
    A = np.zeros((3 * plan.n_obs, 3 * plan.n_obs))
    for b in range(plan.band.shape[0]):
        lo, hi = plan.offsets[b], plan.offsets[b + 1]
        T = toeplitz_dense(plan.band[b], hi - lo)
        Pb = Pd[lo:hi]
        A += Pb.T @ (T @ Pb)
    return A


def dense_solve(plan: OraclePlan, b) -> np.ndarray:
    """m* = A^-1 b by a dense Cholesky factorisation (tiny only)."""
    A = dense_A(plan)
    c = scipy.linalg.cho_factor(A)
    return scipy.linalg.cho_solve(c, np.asarray(b, dtype=np.float64).reshape(-1)).reshape(-1, 3)


# ------------------------------------------------------------------------------------------
# Algorithm 2 (block form, Orthomin) applied to s right-hand sides
# ------------------------------------------------------------------------------------------


def _pivoted_cholesky(G, tol):
    """Rank-revealing Cholesky G[piv][:, piv] ~= L L^T; returns (L, piv, rank)."""
    G = np.array(G, dtype=np.float64)
    n = G.shape[0]
    piv = np.arange(n)
    L = np.zeros_like(G)
    scale = max(float(np.max(np.abs(np.diag(G)))), 1e-300)
    rank = n
    for k in range(n):
        d = np.diag(G)[k:] - np.sum(L[k:, :k] ** 2, axis=1)
        j = k + int(np.argmax(d))
        if d[j - k] <= tol * scale:
            rank = k
            break
        if j != k:
            G[[k, j]] = G[[j, k]]
            G[:, [k, j]] = G[:, [j, k]]
            L[[k, j]] = L[[j, k]]
            piv[[k, j]] = piv[[j, k]]
        L[k, k] = math.sqrt(d[j - k])
        L[k + 1:, k] = (G[k + 1:, k] - L[k + 1:, :k] @ L[k, :k]) / L[k, k]
    return L[:rank, :rank], piv[:rank], rank


@dataclass
class BlockCGResult:
    X: np.ndarray           # [s, n_obs, 3]
    iters: int
    converged: np.ndarray   # [s]
    rel_res: np.ndarray     # [s]


def block_cg(plan: OraclePlan, Bm, tol: float = 1e-6, max_iter: int = 10000,
             rank_tol: float = 1e-12, apply=None) -> BlockCGResult:
    """Algorithm 2 (Orthomin) with R_0 = [b_1 .. b_s] (s independent right-hand sides).

    P_k = Z_k (Z_k^T A Z_k)^{-1/2} with the inverse square root taken as the Cholesky factor
    (Sect. 3.2: "computed using a Cholesky factorization"), alpha_k = P_k^T R_{k-1},
    X_k = X_{k-1} + P_k alpha_k, R_k = R_{k-1} - A P_k alpha_k,
    Z_{k+1} = (I - P_k P_k^T A) M R_k.  Column j counts as converged once
    ||R_j|| < eps ||b_j||; the search block is built from the unconverged columns only and
    dependent directions are dropped by a pivoted Cholesky (the paper leaves this case open).
    """
    A = apply if apply is not None else (lambda v: apply_A(plan, v))
    Bm = np.asarray(Bm, dtype=np.float64).reshape(Bm.shape[0], -1)   # [s, n]
    s, n = Bm.shape
    X = np.zeros_like(Bm)
    R = Bm.copy()
    bn = np.linalg.norm(Bm, axis=1)
    bn_safe = np.where(bn > 0, bn, 1.0)
    conv = bn == 0
    MR = lambda Rc: np.stack([precond_bd(plan, r.reshape(-1, 3)).reshape(-1) for r in Rc])
    Ablk = lambda Zc: np.stack([A(z.reshape(-1, 3)).reshape(-1) for z in Zc])
    Z = MR(R[~conv])
    k = 0
    rel = np.linalg.norm(R, axis=1) / bn_safe
    while k < max_iter and not conv.all() and Z.shape[0] > 0:
        AZ = Ablk(Z)
        G = Z @ AZ.T                                   # Z^T A Z  (t x t)
        G = 0.5 * (G + G.T)
        L, piv, rank = _pivoted_cholesky(G, rank_tol)
        if rank == 0:
            break
        Linv = scipy.linalg.solve_triangular(L, np.eye(rank), lower=True)   # L^-1
        P = Linv @ Z[piv]                              # rows = columns of P_k = Z L^-T
        AP = Linv @ AZ[piv]
        alpha = P @ R.T                                # P_k^T R_{k-1}  (rank x s)
        X = X + alpha.T @ P
        R = R - alpha.T @ AP
        k += 1
        rel = np.linalg.norm(R, axis=1) / bn_safe
        conv = conv | (rel < tol)
        if conv.all():
            break
        W = MR(R[~conv])
        Z = W - (W @ AP.T) @ P                         # (I - P P^T A) M R
    return BlockCGResult(X=X.reshape(s, -1, 3), iters=k, converged=conv, rel_res=rel)


def ecg_split(b, t: int) -> np.ndarray:
    """Split of a residual into t columns that sum to it (Sect. 3.2, ECG): column i keeps the
    unknowns of the pixels p with floor(p t / n_obs) = i (contiguous ranges of compacted pixels,
    all three Stokes parameters of a pixel in the same subdomain) and is zero elsewhere."""
    b = np.asarray(b, dtype=np.float64).reshape(-1, 3)
    n = b.shape[0]
    dom = (np.arange(n, dtype=np.int64) * t) // n
    R = np.zeros((t, n, 3))
    R[dom, np.arange(n)] = b
    return R


@dataclass
class ECGResult:
    x: np.ndarray           # [n_obs, 3], the sum of the t columns of X
    iters: int
    converged: bool
    rel_res: float          # ||sum_i R_k^(i)|| / ||b||
    iterates: Optional[list] = None
    galerkin: Optional[list] = None   # max |P_k^T R_k| / ||b|| per iteration


def ecg(plan: OraclePlan, b, t: int, tol: float = 1e-6, max_iter: int = 10000,
        variant: str = "orthomin", rank_tol: float = 1e-12, keep_iterates: bool = False,
        apply=None) -> ECGResult:
    """Enlarged CG (Sect. 3.2, the ECG algorithm) for one right-hand side, x_0 = 0.

    r_0 = b is split into t columns R_0 (ecg_split) with sum_i R_0^(i) = r_0; Z_1 = M R_0; then
    P_k = Z_k (Z_k^T A Z_k)^{-1/2} (inverse Cholesky factor, dependent directions dropped by a
    pivoted Cholesky), alpha_k = P_k^T R_{k-1}, X_k = X_{k-1} + P_k alpha_k,
    R_k = R_{k-1} - A P_k alpha_k, stop when ||sum_i R_k^(i)|| < eps ||b||, and
        Orthomin: Z_{k+1} = (I - P_k P_k^T A) M R_k,
        Orthodir: Z_{k+1} = (I - P_k P_k^T A - P_{k-1} P_{k-1}^T A) M A P_k.
    The answer is x_k = sum_i X_k^(i).  ``iters`` counts block A-applications.
    """
    if variant not in ("orthomin", "orthodir"):
        raise ValueError("variant must be 'orthomin' or 'orthodir'")
    A = apply if apply is not None else (lambda v: apply_A(plan, v))
    b = np.asarray(b, dtype=np.float64).reshape(-1, 3)
    n = b.shape[0]
    bnorm = float(np.linalg.norm(b))
    if bnorm == 0.0:
        return ECGResult(x=np.zeros_like(b), iters=0, converged=True, rel_res=0.0)
    R = ecg_split(b, t).reshape(t, -1)                 # rows = columns of R
    X = np.zeros_like(R)
    MR = lambda Rc: np.stack([precond_bd(plan, r.reshape(-1, 3)).reshape(-1) for r in Rc])
    Ablk = lambda Zc: np.stack([A(z.reshape(-1, 3)).reshape(-1) for z in Zc])
    Z = MR(R)
    P_prev = AP_prev = None
    its = [] if keep_iterates else None
    gal = []
    k = 0
    rel = 1.0
    converged = False
    while k < max_iter and Z.shape[0] > 0:
        AZ = Ablk(Z)
        G = Z @ AZ.T                                   # Z^T A Z
        G = 0.5 * (G + G.T)
        L, piv, rank = _pivoted_cholesky(G, rank_tol)
        if rank == 0:
            break
        Linv = scipy.linalg.solve_triangular(L, np.eye(rank), lower=True)
        P = Linv @ Z[piv]                              # P_k = Z L^-T (rows)
        AP = Linv @ AZ[piv]
        alpha = P @ R.T                                # P_k^T R_{k-1}  (rank x t)
        X = X + alpha.T @ P
        R = R - alpha.T @ AP
        k += 1
        gal.append(float(np.max(np.abs(P @ R.T))) / bnorm)
        rel = float(np.linalg.norm(R.sum(axis=0))) / bnorm
        if keep_iterates:
            its.append(X.sum(axis=0).reshape(-1, 3).copy())
        if rel < tol:
            converged = True
            break
        if variant == "orthomin":
            W = MR(R)
            Z = W - (W @ AP.T) @ P
        else:
            W = MR(AP)
            Z = W - (W @ AP.T) @ P
            if P_prev is not None:
                Z = Z - (W @ AP_prev.T) @ P_prev
        P_prev, AP_prev = P, AP
    return ECGResult(x=X.sum(axis=0).reshape(-1, 3), iters=k, converged=converged, rel_res=rel,
                     iterates=its, galerkin=gal)


# ------------------------------------------------------------------------------------------
# Algorithm 3 (Lanczos) and the two-level a-posteriori preconditioner (Sect. 3.2)
# ------------------------------------------------------------------------------------------


def lanczos(plan: OraclePlan, b, m: int, eps: float = np.finfo(np.float64).eps, apply=None):
    """Algorithm 3 on A (not M_BD A), x_0 = 0 so v_1 = b / ||b||; no re-orthogonalisation.

    Returns (T_m [m x m], V_m [n x m], A V_m [n x m], beta_{m+1}, v_{m+1} or None).
    """
    A = apply if apply is not None else (lambda v: apply_A(plan, v))
    r0 = np.asarray(b, dtype=np.float64).reshape(-1)
    beta = float(np.linalg.norm(r0))
    v = r0 / beta
    v_prev = np.zeros_like(v)
    V, AV, alphas, betas = [], [], [], []
    beta_k = 0.0
    v_next = None
    for k in range(m):
        Av = A(v.reshape(-1, 3)).reshape(-1)
        w = Av - beta_k * v_prev
        V.append(v)
        AV.append(Av)
        a = float(np.dot(w, v))
        w = w - a * v
        alphas.append(a)
        beta_next = float(np.linalg.norm(w))
        if beta_next < eps:
            beta_k = beta_next
            v_next = None
            break
        v_prev, v = v, w / beta_next
        betas.append(beta_next)
        beta_k = beta_next
        v_next = v
    mm = len(alphas)
    T = np.diag(alphas)
    off = np.array(betas[: mm - 1])
    if mm > 1:
        T += np.diag(off, 1) + np.diag(off, -1)
    beta_last = betas[mm - 1] if len(betas) >= mm else 0.0
    return T, np.stack(V, axis=1), np.stack(AV, axis=1), beta_last, v_next


@dataclass
class TwoLevel:
    Z: np.ndarray       # [n, k]
    Zp: np.ndarray      # A Z
    E: np.ndarray       # Z^T A Z
    Einv: np.ndarray    # pseudo-inverse of E
    theta: np.ndarray   # Ritz values


def two_level_from_lanczos(plan: OraclePlan, b, m: int, rcond: float = 1e-12,
                           apply=None) -> TwoLevel:
    """A-posteriori deflation space: Ritz vectors Z = V_m X of T_m = X Theta X^T, Z' = (A V_m) X,
    coarse matrix E = Z^T Z' and its SVD pseudo-inverse (singular values below rcond * s_max cut)."""
    T, V, AV, _, _ = lanczos(plan, b, m, apply=apply)
    theta, Xe = np.linalg.eigh(T)
    Z = V @ Xe
    Zp = AV @ Xe
    E = Z.T @ Zp
    Einv = np.linalg.pinv(E, rcond=rcond)
    return TwoLevel(Z=Z, Zp=Zp, E=E, Einv=Einv, theta=theta)


def two_level_apriori(plan: OraclePlan, n_int: int, rcond: float = 1e-12, apply=None) -> TwoLevel:
    """A-priori deflation space (Sect. 3.2, 2lvl a priori construction): one column per time
    interval j (blocks are detector-major, block b belongs to interval b mod n_int).  With s_p^j the
    number of kept samples of pixel p in interval j and s_p their sum, the column's total-intensity
    entry at pixel p is s_p^j / s_p and its Q and U entries are 0, so the I rows of Z are a partition
    of unity.  Z' = A Z, E = Z^T Z', E^-1 its SVD pseudo-inverse; theta is left at 0 (no Ritz
    values)."""
    A = apply if apply is not None else (lambda v: apply_A(plan, v))
    n = plan.n_obs
    s_pj = np.zeros((n, n_int))
    for b in range(plan.block_len.size):
        lp = plan.lpix[plan.offsets[b]:plan.offsets[b + 1]]
        lp = lp[lp >= 0]
        s_pj[:, b % n_int] += np.bincount(lp, minlength=n)
    s_p = s_pj.sum(axis=1)
    Z = np.zeros((n, 3, n_int))
    Z[:, 0, :] = s_pj / s_p[:, None]
    Z = Z.reshape(3 * n, n_int)
    Zp = np.stack([A(Z[:, j].reshape(-1, 3)).reshape(-1) for j in range(n_int)], axis=1)
    E = Z.T @ Zp
    Einv = np.linalg.pinv(E, rcond=rcond)
    return TwoLevel(Z=Z, Zp=Zp, E=E, Einv=Einv, theta=np.zeros(n_int))


def precond_2lvl(plan: OraclePlan, tl: TwoLevel, r) -> np.ndarray:
    """Eq. 2lvlDef0: M_2lvl r = M_BD r - M_BD Z' E^-1 Z^T r + Z E^-1 Z^T r (right to left)."""
    r = np.asarray(r, dtype=np.float64).reshape(-1)
    y = tl.Einv @ (tl.Z.T @ r)
    t1 = precond_bd(plan, r.reshape(-1, 3)).reshape(-1)
    t2 = precond_bd(plan, (tl.Zp @ y).reshape(-1, 3)).reshape(-1)
    return (t1 - t2 + tl.Z @ y).reshape(-1, 3)


__all__ += ["precond_2lvl", "BlockCGResult", "apply_A_at_pixels", "ecg_split", "ecg", "ECGResult",
            "two_level_apriori"]


def apply_A_at_pixels(pix, psi, block_off, band, keep, x_glob, pixels, sample_idx=None):
    """(A x)_p for a few global pixels p, one by one, for problems too large for `apply_A`.

    Definitions of Sect. 3.2 evaluated at the samples t that hit p (mask G from `keep`):
    y_t = sum_{|k| <= lambda, t+k in block(t)} c_|k| (P~ x)_{t+k}  (Eq. MADCAP), then
    (A x)_p = sum_t w_t y_t.  x_glob is indexed by global pixel ([n_pix, 3]); samples of pixels
    with keep = False, and gaps, are masked on both sides.  `sample_idx[i]` (optional) lists the
    samples of pixels[i].  Returns values [len(pixels), 3] and, per pixel, the sum of the absolute
    values of the terms (the scale against which rounding errors are judged).
    """
    pix = np.asarray(pix)
    block_off = np.asarray(block_off, dtype=np.int64)
    band = np.asarray(band, dtype=np.float64)
    lam = band.shape[1] - 1
    out = np.zeros((len(pixels), 3))
    scale = np.zeros(len(pixels))
    kk = np.arange(-lam, lam + 1)
    for i, p in enumerate(pixels):
        S = np.nonzero(pix == p)[0] if sample_idx is None else np.asarray(sample_idx[i])
        b = np.searchsorted(block_off, S, side="right") - 1
        lo, hi = block_off[b], block_off[b + 1]
        W = S[:, None] + kk[None, :]                       # band windows
        inb = (W >= lo[:, None]) & (W < hi[:, None])
        Wc = np.clip(W, 0, pix.size - 1)
        pw = pix[Wc]
        ok = inb & (pw >= 0)
        ok &= np.where(pw >= 0, keep[np.clip(pw, 0, None)], False)
        wgt = pointing_weights(np.asarray(psi)[Wc.ravel()]).reshape(W.shape + (3,))
        xm = x_glob[np.clip(pw, 0, None)]
        t = np.where(ok, (wgt * xm).sum(axis=2), 0.0)      # (P~ x) on the windows
        c = band[b][:, np.abs(kk)]                         # c_|k| of each sample's block
        y = (c * t).sum(axis=1)
        wt = pointing_weights(np.asarray(psi)[S])
        out[i] = (wt * y[:, None]).sum(axis=0)
        scale[i] = (np.abs(c * t).sum(axis=1)[:, None] * np.abs(wt)).sum()
    return out, scale


def cpu_threads() -> int:
    return len(os.sched_getaffinity(0))


# ------------------------------------------------------------------------------------------
# noise weights from the data (Sect. 2.2, the MAPPRAISER weights paragraph; Eq. noisepowermodel)
# ------------------------------------------------------------------------------------------

NOISE_SEG = 32768   # periodogram segment and inverse-FFT length (frequencies k / NOISE_SEG)


def periodogram(d, pix, block_len, seg: int = NOISE_SEG):
    """Averaged periodogram of each block's gap-masked TOD G d ("the average periodogram of each
    detector time stream").  A block of n samples gives max(1, floor(n / seg)) segments of seg
    samples (one zero-padded segment when n < seg; a partial last segment is left out).  For each
    segment P_k = |X_k|^2 / n_kept (X = real DFT of the seg samples, n_kept = kept samples in the
    segment), averaged over the segments, k = 0..seg/2, frequency k / seg cycles per sample; white
    noise of variance s^2 then has E P_k = s^2.  Returns (P [n_blocks, seg/2 + 1], segments used)."""
    d = np.asarray(d, dtype=np.float64)
    pix = np.asarray(pix)
    off = block_offsets(block_len)
    nb = len(block_len)
    P = np.zeros((nb, seg // 2 + 1))
    nseg = np.zeros(nb, dtype=np.int64)
    for b in range(nb):
        n = int(off[b + 1] - off[b])
        gd = np.where(pix[off[b]:off[b + 1]] >= 0, d[off[b]:off[b + 1]], 0.0)
        kept = pix[off[b]:off[b + 1]] >= 0
        count = max(1, n // seg) if n > 0 else 0
        used = 0
        for s_ in range(count):
            x = np.zeros(seg)
            m = min(seg, n - s_ * seg)
            x[:m] = gd[s_ * seg:s_ * seg + m]
            nk = int(np.count_nonzero(kept[s_ * seg:s_ * seg + m]))
            if nk == 0:
                continue
            P[b] += np.abs(np.fft.rfft(x)) ** 2 / nk
            used += 1
        if used:
            P[b] /= used
        nseg[b] = used
    return P, nseg


def psd_model(f, theta):
    """Eq. noisepowermodel with f_0 = 0: P(f) = sigma^2 (1 + (f_knee / f)^alpha), theta =
    (log sigma^2, log f_knee, alpha), f and f_knee in cycles per sample."""
    ls2, lfk, a = theta
    return np.exp(ls2) * (1.0 + np.exp(a * (lfk - np.log(f))))


def psd_fit_init(P, seg: int = NOISE_SEG):
    """Starting point of the fit: sigma^2 = mean of the upper half of the band (k >= seg/4); over
    the bins with P_k > 3 sigma^2, a straight line through log(P_k / sigma^2 - 1) against log f
    gives slope -alpha and intercept alpha log f_knee (alpha clipped to [0.2, 5]); with fewer than
    three such bins alpha = 1 and f_knee = 1 / seg."""
    P = np.asarray(P, dtype=np.float64)
    k = np.arange(P.size)
    s2 = float(np.mean(P[seg // 4:]))
    sel = (k >= 1) & (P > 3.0 * s2)
    if np.count_nonzero(sel) >= 3:
        x = np.log(k[sel] / seg)
        y = np.log(P[sel] / s2 - 1.0)
        slope, icpt = np.polyfit(x, y, 1)
        a = float(np.clip(-slope, 0.2, 5.0))
        lfk = icpt / a
    else:
        a, lfk = 1.0, math.log(1.0 / seg)
    return np.array([math.log(s2), lfk, a])


def fit_psd(P, seg: int = NOISE_SEG):
    """Least-squares fit of log P_k by log P(f_k; theta) over k = 1..seg/2 (the periodogram's
    spread is multiplicative, so residuals are taken in log space), Levenberg-Marquardt from
    psd_fit_init.  Returns theta = (log sigma^2, log f_knee, alpha)."""
    P = np.asarray(P, dtype=np.float64)
    k = np.arange(1, P.size)
    f = k / seg
    y = np.log(P[1:])
    res = scipy.optimize.least_squares(lambda th: y - np.log(psd_model(f, th)), psd_fit_init(P, seg),
                                       method="lm", xtol=1e-15, ftol=1e-15, gtol=1e-15, max_nfev=20000)
    return res.x


def band_from_psd(theta, lam: int, seg: int = NOISE_SEG):
    """First row of the inverse-noise Toeplitz block from a fitted PSD: 1/P(f_k) on the seg-point
    grid (1/P(0) := 0), inverse real DFT, Gaussian window N(0, lambda/2) on the lags, cut at
    lambda (Sect. 2.2: "smoothed with a gaussian window ... and cut at the a priori specified half
    bandwidth")."""
    f = np.arange(seg // 2 + 1) / seg
    S = np.zeros(f.size)
    S[1:] = 1.0 / psd_model(f[1:], theta)
    c = np.fft.irfft(S, n=seg)[:lam + 1]
    if lam > 0:
        tau = np.arange(lam + 1)
        c = c * np.exp(-0.5 * (tau / (lam / 2.0)) ** 2)
    return c


def estimate_bands(d, pix, block_len, lam: int, seg: int = NOISE_SEG):
    """The weights of each block from its own data: periodogram, fit, inverse band.  Returns
    (bands [n_blocks, lam + 1], theta [n_blocks, 3]); blocks without a kept sample get zeros."""
    P, nseg = periodogram(d, pix, block_len, seg)
    nb = len(block_len)
    bands = np.zeros((nb, lam + 1))
    th = np.zeros((nb, 3))
    for b in range(nb):
        if nseg[b] == 0:
            continue
        th[b] = fit_psd(P[b], seg)
        bands[b] = band_from_psd(th[b], lam, seg)
    return bands, th


__all__ += ["NOISE_SEG", "periodogram", "psd_model", "psd_fit_init", "fit_psd", "band_from_psd",
            "estimate_bands"]


# ------------------------------------------------------------------------------------------
# template map-making with diagonal weights (Sect. 2, Eq. genMapEstimator with the filtering
# operator F_T; the templates of Appendix A)
# ------------------------------------------------------------------------------------------


@dataclass
class Templates:
    """Template classes of every block (detector x stationary interval): n_poly Legendre orders,
    n_az azimuth bins (or interpolation nodes when interp), n_hwp harmonics of the HWP angle."""

    n_poly: int = 0
    n_az: int = 0
    n_hwp: int = 0
    interp: bool = False

    @property
    def k(self) -> int:
        return self.n_poly + self.n_az + 2 * self.n_hwp


def template_matrix(n: int, az, hwp, kept, tm: Templates) -> np.ndarray:
    """The templates of one block of n samples as columns [n, K] (Appendix A), one interval per
    block:
      Legendre P_k(x), k < n_poly, at x = 2 tau / (n - 1) - 1 (x = 0 when n = 1), rescaled by
      sqrt((2k + 1) / n) so that the columns are orthonormal up to the discretisation;
      azimuth: the grid spans [min, max] of az over the block's kept samples; binned: value 1 in
      bin floor((az - lo) / (hi - lo) n_az) (clamped to n_az - 1; bin 0 when hi = lo); interpolated:
      nodes lo + i (hi - lo) / (n_az - 1), the two nodes bracketing az get (phi_{i+1} - az) / step
      and (az - phi_i) / step (node 0 alone when hi = lo or n_az = 1);
      HWP: cos(k phi), sin(k phi), k = 1..n_hwp.
    Rows of masked samples are kept (the weights zero them)."""
    az = np.asarray(az, dtype=np.float64)
    hwp = np.asarray(hwp, dtype=np.float64)
    T = np.zeros((n, tm.k))
    tau = np.arange(n)
    x = 2.0 * tau / (n - 1) - 1.0 if n > 1 else np.zeros(n)
    for k in range(tm.n_poly):
        T[:, k] = scipy.special.eval_legendre(k, x) * math.sqrt((2 * k + 1) / n)
    c0 = tm.n_poly
    if tm.n_az > 0:
        sel = np.asarray(kept, dtype=bool)
        lo = float(az[sel].min()) if sel.any() else 0.0
        hi = float(az[sel].max()) if sel.any() else 0.0
        if tm.interp:
            if hi > lo and tm.n_az > 1:
                step = (hi - lo) / (tm.n_az - 1)
                pos = np.clip((az - lo) / step, 0.0, tm.n_az - 1)
                i = np.minimum(np.floor(pos).astype(np.int64), tm.n_az - 2)
                frac = pos - i
                T[tau, c0 + i] = 1.0 - frac
                T[tau, c0 + i + 1] = frac
            else:
                T[:, c0] = 1.0
        else:
            if hi > lo:
                b = np.floor((az - lo) / (hi - lo) * tm.n_az).astype(np.int64)
                b = np.clip(b, 0, tm.n_az - 1)
            else:
                b = np.zeros(n, dtype=np.int64)
            T[tau, c0 + b] = 1.0
    c0 += tm.n_az
    for k in range(1, tm.n_hwp + 1):
        T[:, c0 + 2 * (k - 1)] = np.cos(k * hwp)
        T[:, c0 + 2 * (k - 1) + 1] = np.sin(k * hwp)
    return T


def template_filter(plan: OraclePlan, weights, tm: Templates, az, hwp, v, rcond: float = 1e-12) -> np.ndarray:
    """F_T v = W v - W T (T^T W T)^+ T^T W v block by block (Sect. 2, Eq. genMapEstimator; the
    kernel inverted by SVD with singular values below rcond of the largest dropped, as the templates
    package does), W = diag(w_b) on the kept samples of block b and 0 on masked ones (G)."""
    v = np.asarray(v, dtype=np.float64)
    out = np.zeros_like(v)
    for b in range(plan.block_len.size):
        lo, hi = plan.offsets[b], plan.offsets[b + 1]
        n = int(hi - lo)
        if n == 0:
            continue
        kept = plan.lpix[lo:hi] >= 0
        w = np.where(kept, float(weights[b]), 0.0)
        wv = w * v[lo:hi]
        if tm.k == 0:
            out[lo:hi] = wv
            continue
        T = template_matrix(n, az[lo:hi], hwp[lo:hi], kept, tm)
        K = T.T @ (w[:, None] * T)
        c = np.linalg.pinv(K, rcond=rcond, hermitian=True) @ (T.T @ wv)
        out[lo:hi] = wv - w * (T @ c)
    return out


def apply_A_templates(plan: OraclePlan, weights, tm: Templates, az, hwp, x) -> np.ndarray:
    """A x = P~^T F_T P~ x."""
    return point(plan, template_filter(plan, weights, tm, az, hwp, unpoint(plan, x)))


def rhs_templates(plan: OraclePlan, weights, tm: Templates, az, hwp, d) -> np.ndarray:
    """b = P~^T F_T G d (F_T carries the mask)."""
    return point(plan, template_filter(plan, weights, tm, az, hwp, np.asarray(d, dtype=np.float64)))


__all__ += ["Templates", "template_matrix", "template_filter", "apply_A_templates", "rhs_templates"]
