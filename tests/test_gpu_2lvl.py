"""Two-level a-posteriori preconditioner (Lanczos, Algorithm 3; A-DEF1, Eq. 2lvlDef0) on the GPU
against the FP64 oracle.  Z and Z' are stored in FP32 on the device, so identities that hold
exactly in the oracle hold here to ~1e-5 relative."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from gpu_helpers import cuda, mm, plans

pytestmark = pytest.mark.gpu

M = 8


@pytest.fixture(scope="module")
def tiny():
    cfg = synth.tiny_config()
    prob = synth.make_ground_problem(cfg)
    gp, op, nb = plans(prob)
    b = O.rhs(op, nb["d"])
    mm().mm_deflation_build(gp, cuda(b), M, precision=0)
    return cfg, gp, op, b


def test_ritz_values_match_oracle_lanczos(tiny):
    cfg, gp, op, b = tiny
    k, Z, theta = mm().mm_deflation_get(gp)
    tl = O.two_level_from_lanczos(op, b, M)
    assert k == M
    np.testing.assert_allclose(np.sort(theta), np.sort(tl.theta), rtol=1e-7)
    # Ritz vectors agree up to sign (FP32 storage of Z)
    Zo = tl.Z.T.reshape(M, -1, 3)
    Zg = Z.cpu().numpy()
    og = np.argsort(theta)
    oo = np.argsort(tl.theta)
    for i, j in zip(og, oo):
        a, c = Zg[i].ravel(), Zo[j].ravel()
        cos = abs(np.dot(a, c)) / (np.linalg.norm(a) * np.linalg.norm(c))
        assert cos > 1 - 1e-6


def test_two_level_maps_A_Z_to_Z(tiny):
    # (I - AQ) A Z = 0 and the second level give M_2lvl A Z = Z (Eq. 2lvlDef)
    cfg, gp, op, b = tiny
    k, Z, theta = mm().mm_deflation_get(gp)
    AZ = torch.empty_like(Z)
    mm().mm_apply_A(gp, Z.contiguous(), AZ)
    out = torch.empty_like(Z)
    mm().mm_deflation_apply(gp, AZ, out)
    for j in range(k):
        err = float((out[j] - Z[j]).norm() / Z[j].norm())
        assert err < 1e-4, (j, err)


@pytest.mark.parametrize("precision", [0, 1])
def test_two_level_pcg_converges_faster_and_matches(tiny, precision):
    cfg, gp, op, b = tiny
    x_bd = torch.empty(op.n_obs, 3, dtype=torch.float64, device="cuda")
    x_2l = torch.empty_like(x_bd)
    i_bd = mm().mm_pcg_solve(gp, cuda(b), x_bd, tol=1e-8, precision=precision)[0]
    i_2l = mm().mm_pcg_solve(gp, cuda(b), x_2l, tol=1e-8, precision=precision,
                             precond=mm().MM_PREC_2LVL_POST)[0]
    # n_iter(2lvl) <= n_iter(BD) (Sect. 3.2); the FP32 path restarts at its FP64 residual checks
    assert i_2l.status == 0 and i_2l.iters <= i_bd.iters + (3 if precision else 0)
    m_ref = O.pcg(op, b, tol=1e-12, max_iter=10000).x
    tl = O.two_level_from_lanczos(op, b, M)
    o2 = O.pcg(op, b, tol=1e-8, precond=lambda r: O.precond_2lvl(op, tl, r))
    err_or = np.linalg.norm(o2.x - m_ref) / np.linalg.norm(m_ref)
    err = np.linalg.norm(x_2l.cpu().numpy() - m_ref) / np.linalg.norm(m_ref)
    assert err <= 10 * err_or + 1e-9, (err, err_or)
    if precision == 0:
        assert abs(i_2l.iters - o2.iters) <= 2
    assert i_2l.true_rel_res < 1e-8
