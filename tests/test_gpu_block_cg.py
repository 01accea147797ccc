"""Block CG (Algorithm 2, block Orthomin form on s right-hand sides) against the FP64 oracle.

Search blocks are FP32 on the GPU, so iterates differ from the oracle's FP64 block CG at the
1e-6 level; converged maps are compared with the oracle's PCG solutions of each column at the
mixed-precision tolerance (rel. map error <= 1e-5) and every column's FP64 true residual must be
below tol.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from gpu_helpers import cuda, mm, plans

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tiny():
    cfg = synth.tiny_config()
    prob = synth.make_ground_problem(cfg, n_real=5)
    gp, op, nb = plans(prob, precision=1)
    B = np.stack([O.rhs(op, nb["d"][j]) for j in range(5)])
    refs = [O.pcg(op, B[j], tol=1e-8, max_iter=5000) for j in range(5)]
    return cfg, gp, op, B, refs


@pytest.mark.parametrize("precision", [1, 0])
def test_block_cg_s1_matches_pcg(tiny, precision):
    cfg, gp, op, B, refs = tiny
    x = torch.empty(1, op.n_obs, 3, dtype=torch.float64, device="cuda")
    info = mm().mm_block_cg_solve(gp, cuda(B[:1]), x, block_width=1, tol=1e-8, precision=precision)[0]
    assert info.status == 0 and info.true_rel_res < 1e-8
    assert abs(info.iters - refs[0].iters) <= max(3, refs[0].iters // 10)
    err = np.linalg.norm(x[0].cpu().numpy() - refs[0].x) / np.linalg.norm(refs[0].x)
    assert err <= 1e-5, err


@pytest.mark.parametrize("width", [0, 2, 4])
def test_block_cg_multi_rhs_matches_oracle(tiny, width):
    cfg, gp, op, B, refs = tiny
    x = torch.empty(5, op.n_obs, 3, dtype=torch.float64, device="cuda")
    infos = mm().mm_block_cg_solve(gp, cuda(B), x, block_width=width, tol=1e-8)
    for j in range(5):
        assert infos[j].status == 0 and infos[j].true_rel_res < 1e-8
        err = np.linalg.norm(x[j].cpu().numpy() - refs[j].x) / np.linalg.norm(refs[j].x)
        assert err <= 1e-5, (j, err)
    if width in (0, 4):   # a shared block never needs more iterations than its slowest column's PCG
        assert max(i.iters for i in infos[:4]) <= max(r.iters for r in refs[:4]) + 2


def test_block_cg_oracle_iterates_agree(tiny):
    # the oracle's own block CG (FP64) on the same block converges in a similar iteration count
    cfg, gp, op, B, refs = tiny
    ob = O.block_cg(op, B[:4], tol=1e-8, max_iter=2000)
    x = torch.empty(4, op.n_obs, 3, dtype=torch.float64, device="cuda")
    infos = mm().mm_block_cg_solve(gp, cuda(B[:4]), x, block_width=4, tol=1e-8)
    assert ob.converged.all()
    assert abs(max(i.iters for i in infos) - ob.iters) <= max(3, ob.iters // 5)
    for j in range(4):
        assert np.linalg.norm(x[j].cpu().numpy() - ob.X[j]) <= 1e-5 * np.linalg.norm(ob.X[j])


def test_block_cg_zero_column_and_max_iter(tiny):
    cfg, gp, op, B, refs = tiny
    Bz = B[:3].copy()
    Bz[1] = 0.0
    x = torch.empty(3, op.n_obs, 3, dtype=torch.float64, device="cuda")
    infos = mm().mm_block_cg_solve(gp, cuda(Bz), x, block_width=3, tol=1e-8)
    assert infos[1].status == 0 and float(x[1].abs().max()) == 0.0
    infos = mm().mm_block_cg_solve(gp, cuda(B[:2]), x[:2].contiguous(), block_width=2, tol=1e-14,
                                   max_iter=3, raise_on_error=False)
    assert all(i.status == mm().MM_ENOTCONV for i in infos)
