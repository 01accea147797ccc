"""mm_pcg_solve replays a captured CUDA graph across calls; the graph holds raw pointers to plan
buffers that other calls may reallocate (the un-pointed t buffers grow with the number of
right-hand sides; a deflation build replaces the space).  Each case interleaves such a call
between solves and checks the later solve against the oracle."""
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
    prob = synth.make_ground_problem(cfg)
    _, op, nb = plans(prob)
    b = O.rhs(op, nb["d"])
    ref = O.pcg(op, b, tol=1e-10, max_iter=5000)
    return cfg, prob, op, b, ref


@pytest.mark.parametrize("plan_prec,solve_prec", [(3, 1), (3, 0), (2, 0), (1, 1)])
def test_solve_after_buffers_grew(tiny, plan_prec, solve_prec):
    cfg, prob, op, b, ref = tiny
    gp, _, _ = plans(prob, precision=plan_prec)
    x = torch.empty(op.n_obs, 3, dtype=torch.float64, device="cuda")
    i1 = mm().mm_pcg_solve(gp, cuda(b), x, tol=cfg.tol, precision=solve_prec)[0]
    x1 = x.cpu().numpy()
    # three right-hand sides grow the plan's t buffers (FP32 and df64)
    X = cuda(np.random.default_rng(1).standard_normal((3, op.n_obs, 3)))
    Y = torch.empty_like(X)
    mm().mm_apply_A(gp, X, Y)
    mm().mm_rhs(gp, cuda(np.stack([prob.d.cpu().numpy()] * 3)), Y)
    x.zero_()
    i2 = mm().mm_pcg_solve(gp, cuda(b), x, tol=cfg.tol, precision=solve_prec)[0]
    # the P^T atomics make runs differ in the last bits; the FP64-class solves stay in step
    assert i1.status == 0 and i2.status == 0
    if solve_prec == 0:
        assert abs(i1.iters - i2.iters) <= 1
    x2 = x.cpu().numpy()
    assert np.linalg.norm(x2 - x1) <= 1e-6 * np.linalg.norm(x1)
    assert np.linalg.norm(x2 - ref.x) <= 1e-5 * np.linalg.norm(ref.x)


def test_two_level_solve_after_space_rebuilt(tiny):
    cfg, prob, op, b, ref = tiny
    gp, _, _ = plans(prob, precision=3)
    x = torch.empty(op.n_obs, 3, dtype=torch.float64, device="cuda")
    mm().mm_deflation_build_apriori(gp, precision=1)
    mm().mm_pcg_solve(gp, cuda(b), x, tol=cfg.tol, precision=1, precond=1)
    mm().mm_deflation_build(gp, cuda(b), 8, precision=0)          # a larger space, new buffers
    x.zero_()
    info = mm().mm_pcg_solve(gp, cuda(b), x, tol=cfg.tol, precision=1, precond=1)[0]
    tl = O.two_level_from_lanczos(op, b, 8)
    two = O.pcg(op, b, tol=cfg.tol, max_iter=5000, precond=lambda r: O.precond_2lvl(op, tl, r))
    assert info.status == 0 and info.iters <= 2 * two.iters + 4
    assert np.linalg.norm(x.cpu().numpy() - ref.x) <= 1e-5 * np.linalg.norm(ref.x)
    mm().mm_deflation_build_apriori(gp, precision=0)               # and back to the small one
    x.zero_()
    info = mm().mm_pcg_solve(gp, cuda(b), x, tol=cfg.tol, precision=1, precond=1)[0]
    assert info.status == 0
    assert np.linalg.norm(x.cpu().numpy() - ref.x) <= 1e-5 * np.linalg.norm(ref.x)


def test_block_cg_and_ecg_graphs_after_buffers_grew(tiny):
    """The FP32 block CG and enlarged CG replay captured graphs of their iterations, keyed by shape;
    growing the plan's FP32 buffers between solves (more right-hand sides through mm_apply_A)
    must make them capture again rather than replay stale pointers."""
    cfg, prob, op, b, ref = tiny
    m = mm()
    gp, _, _ = plans(prob, precision=3)
    B = cuda(np.stack([b, 2.0 * b, -0.5 * b]))
    X = torch.empty_like(B)
    m.mm_block_cg_solve(gp, B, X, tol=cfg.tol, max_iter=5000)
    X1 = X.cpu().numpy()
    x = torch.empty(op.n_obs, 3, dtype=torch.float64, device="cuda")
    m.mm_ecg_solve(gp, cuda(b), x, 4, tol=cfg.tol, max_iter=5000)
    e1 = x.cpu().numpy()
    W = cuda(np.random.default_rng(2).standard_normal((6, op.n_obs, 3)))
    m.mm_apply_A(gp, W, torch.empty_like(W))          # six columns: larger FP32 t and u buffers
    X.zero_()
    infos = m.mm_block_cg_solve(gp, B, X, tol=cfg.tol, max_iter=5000)
    assert all(i.status == 0 for i in infos)
    for j, s in enumerate((1.0, 2.0, -0.5)):
        assert np.linalg.norm(X[j].cpu().numpy() - s * ref.x) <= 1e-5 * abs(s) * np.linalg.norm(ref.x)
        assert np.linalg.norm(X[j].cpu().numpy() - X1[j]) <= 1e-6 * abs(s) * np.linalg.norm(ref.x)
    x.zero_()
    info = m.mm_ecg_solve(gp, cuda(b), x, 4, tol=cfg.tol, max_iter=5000)
    assert info.status == 0
    assert np.linalg.norm(x.cpu().numpy() - ref.x) <= 1e-5 * np.linalg.norm(ref.x)
    assert np.linalg.norm(x.cpu().numpy() - e1) <= 1e-6 * np.linalg.norm(ref.x)
