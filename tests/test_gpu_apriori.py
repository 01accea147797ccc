"""Two-level a-priori deflation space (Sect. 3.2) on the GPU against the FP64 oracle: one column
per stationary interval holding the fraction of each pixel's kept hits in that interval (I rows),
then the same A-DEF1 preconditioner as the a-posteriori space.  Z and Z' are FP32 on the device."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from gpu_helpers import cuda, mm, plans

pytestmark = pytest.mark.gpu


def multi_interval(seed=3, n_det=2, n_int=3, lam=512):
    lens = [40000, 30000, 20000, 35000, 25000, 15000][: n_det * n_int]
    prob = synth.random_problem(n_det * n_int, lens, 300, lam, seed, gap_frac=0.02, f_knee=5.0,
                                alpha=1.5, hits_per_pix_min=4)
    prob.n_det, prob.n_int = n_det, n_int
    return prob


@pytest.fixture(scope="module")
def mi():
    prob = multi_interval()
    gp, op, nb = plans(prob, precision=3)
    b = O.rhs(op, nb["d"])
    tl = O.two_level_apriori(op, prob.n_int)
    return prob, gp, op, b, tl


@pytest.mark.parametrize("precision", [0, 1])
def test_apriori_space_matches_oracle(mi, precision):
    prob, gp, op, b, tl = mi
    mm().mm_deflation_build_apriori(gp, precision=precision)
    k, Z, theta = mm().mm_deflation_get(gp)
    assert k == prob.n_int and np.all(theta == 0)
    Zo = tl.Z.T.reshape(k, -1, 3)
    np.testing.assert_allclose(Z.cpu().numpy(), Zo, rtol=0, atol=1e-7)
    # M_2lvl A Z = Z through the device's Z' and E^-1
    AZ = torch.empty_like(Z)
    mm().mm_apply_A(gp, Z.contiguous(), AZ)
    out = torch.empty_like(Z)
    mm().mm_deflation_apply(gp, AZ, out)
    for j in range(k):
        assert float((out[j] - Z[j]).norm() / Z[j].norm()) < 1e-4


@pytest.mark.parametrize("precision", [0, 1])
def test_apriori_pcg_matches_oracle(mi, precision):
    prob, gp, op, b, tl = mi
    mm().mm_deflation_build_apriori(gp, precision=0)
    ref = O.pcg(op, b, tol=1e-8, max_iter=5000, precond=lambda r: O.precond_2lvl(op, tl, r))
    bd = O.pcg(op, b, tol=1e-8, max_iter=5000)
    x = torch.empty(op.n_obs, 3, dtype=torch.float64, device="cuda")
    info = mm().mm_pcg_solve(gp, cuda(b), x, tol=1e-8, precision=precision, precond=1)[0]
    assert info.status == 0 and ref.converged
    if precision == 0:
        assert abs(info.iters - ref.iters) <= 2, (info.iters, ref.iters)
    else:
        assert info.iters <= 2 * ref.iters + 4, (info.iters, ref.iters)
    assert ref.iters <= bd.iters + 1
    assert np.linalg.norm(x.cpu().numpy() - ref.x) <= 1e-5 * np.linalg.norm(ref.x)
    assert info.true_rel_res < 1e-8


def test_apriori_single_interval_is_the_monopole():
    cfg = synth.tiny_config()
    prob = synth.make_ground_problem(cfg)
    gp, op, nb = plans(prob, precision=3)
    mm().mm_deflation_build_apriori(gp, precision=1)
    k, Z, _ = mm().mm_deflation_get(gp)
    assert k == 1
    z = Z[0].cpu().numpy()
    np.testing.assert_array_equal(z[:, 0], 1.0)
    np.testing.assert_array_equal(z[:, 1:], 0.0)


def test_apriori_rejects_more_than_64_intervals():
    prob = synth.random_problem(65, [400] * 65, 20, 8, 5, hits_per_pix_min=40)
    prob.n_det, prob.n_int = 1, 65
    gp, _, _ = plans(prob, precision=0)
    with pytest.raises(mm().MMError) as ei:
        mm().mm_deflation_build_apriori(gp)
    assert ei.value.code == 1
