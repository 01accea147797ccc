"""MM_TPLZ_GEMM: the FP32 operators' N^-1 as banded Toeplitz-block GEMMs on the tensor cores
(tcgen05, 3xTF32).  Against the oracle: A x within the FP32 tolerance on ragged blocks (lengths that
are not multiples of the 32-sample rows or the 4096-sample tiles, blocks shorter than one row, an
empty block) for lambda from 0 to 128 (1 to 9 row shifts), several right-hand sides, and a
mixed-precision solve whose map matches the oracle's PCG."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from gpu_helpers import cuda, mm, plans, rel_max

pytestmark = pytest.mark.gpu

BLOCKS = (9000, 5, 4100, 31, 0, 12345)


@pytest.mark.parametrize("lam", [0, 5, 32, 33, 64, 100, 128])
def test_gemm_apply_matches_oracle(lam):
    m = mm()
    prob = synth.random_problem(len(BLOCKS), list(BLOCKS), 200, lam, seed=40 + lam, gap_frac=0.02,
                                hits_per_pix_min=4)
    gp, op, _ = plans(prob, precision=m.MM_FP32_DF64, algo=m.MM_TPLZ_GEMM)
    rng = np.random.default_rng(lam)
    x = cuda(rng.standard_normal((3, op.n_obs, 3)))
    y = torch.empty_like(x)
    m.mm_apply_A(gp, x, y)
    torch.cuda.synchronize()
    xs = x.cpu().numpy()
    ys = y.cpu().numpy()
    for r in range(3):
        assert rel_max(ys[r], O.apply_A(op, xs[r])) < 2e-5, f"column {r}"


def test_gemm_solve_matches_oracle():
    m = mm()
    cfg = synth.tiny_config(lam=96)
    prob = synth.make_ground_problem(cfg)
    gp, op, nb = plans(prob, precision=m.MM_FP32_DF64, algo=m.MM_TPLZ_GEMM)
    ref = O.pcg(op, O.rhs(op, nb["d"]), tol=cfg.tol, max_iter=5000)
    x = torch.empty(op.n_obs, 3, dtype=torch.float64, device="cuda")
    info = m.mm_solve_tod(gp, torch.as_tensor(nb["d"], device="cuda"), x, tol=cfg.tol, max_iter=5000,
                          precision=m.MM_FP32)[0]
    assert info.status == 0 and info.true_rel_res < cfg.tol
    assert np.linalg.norm(x.cpu().numpy() - ref.x) <= 1e-5 * np.linalg.norm(ref.x)


def test_gemm_refused_beyond_its_range():
    m = mm()
    prob = synth.random_problem(2, [5000, 5000], 200, 200, seed=3, hits_per_pix_min=4)
    with pytest.raises(m.MMError) as e:
        plans(prob, precision=m.MM_FP32_DF64, algo=m.MM_TPLZ_GEMM)
    assert e.value.code == m.MM_EINVAL
    prob = synth.random_problem(2, [5000, 5000], 200, 64, seed=3, hits_per_pix_min=4)
    with pytest.raises(m.MMError):
        plans(prob, precision=m.MM_FP64, algo=m.MM_TPLZ_GEMM)
