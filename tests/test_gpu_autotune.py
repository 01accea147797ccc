"""mm_autotune: the tuner times real FP32 A-applications of the plan, keeps the fastest segment
length and window size (the plan's operator stays correct after the rebuild: A x still matches the
oracle within the FP32 tolerance, and a solve still matches it), and its width choice is what
mm_block_cg_solve uses with block_width = 0."""
import numpy as np
import pytest
import torch

import oracle as O
import synth
from gpu_helpers import cuda, mm, plans, rel_max

pytestmark = pytest.mark.gpu


def test_autotune_keeps_operator_and_picks_fastest():
    m = mm()
    cfg = synth.tiny_config(n_det=8, n_samp=131072)
    prob = synth.make_ground_problem(cfg)
    gp, op, nb = plans(prob, precision=m.MM_FP32_DF64)
    res = m.mm_autotune(gp, max_width=8)
    assert res["steps_ms"] and res["win_ms"] and res["width_ms_per_col"]
    assert res["tile_steps"] in res["steps_ms"] and res["win_samples"] in res["win_ms"]
    assert res["steps_ms"][res["tile_steps"]] == min(res["steps_ms"].values())
    assert res["win_ms"][res["win_samples"]] == min(res["win_ms"].values())
    assert all(v > 0 for v in res["win_ms"].values())
    assert res["n_rejected"] == 0 and res["max_rel_dev"] < 2e-5
    best = min(res["width_ms_per_col"].values())
    assert res["width_ms_per_col"][res["block_width"]] <= 1.02 * best + 1e-12
    # the rebuilt operator: A x against the oracle, FP32 tolerance
    rng = np.random.default_rng(1)
    x = cuda(rng.standard_normal((op.n_obs, 3)))
    y = torch.empty_like(x)
    m.mm_apply_A(gp, x, y)
    assert rel_max(y.cpu().numpy(), O.apply_A(op, x.cpu().numpy())) < 2e-5
    # a solve on the tuned plan and the block width it uses
    b = cuda(O.rhs(op, nb["d"]))
    xs = torch.empty_like(b)
    info = m.mm_pcg_solve(gp, b, xs, tol=1e-8, max_iter=5000, precision=m.MM_FP32)[0]
    ref = O.pcg(op, b.cpu().numpy(), tol=1e-8, max_iter=5000)
    assert info.status == 0 and np.linalg.norm(xs.cpu().numpy() - ref.x) <= 1e-5 * np.linalg.norm(ref.x)
    B = torch.stack([b, 2 * b, -b, 0.5 * b, b, b, b, b, b])
    X = torch.empty_like(B)
    infos = m.mm_block_cg_solve(gp, B, X, tol=1e-8, max_iter=5000)
    assert all(i.status == 0 for i in infos)
    w = res["block_width"]
    # the first group holds min(nrhs, w) columns: its A X count equals that of every column in it
    assert len({infos[j].n_apply32 for j in range(min(w, 9))}) == 1


def test_autotune_refuses_fp64_plans():
    m = mm()
    prob = synth.random_problem(2, [20000, 20000], 300, 64, seed=22, hits_per_pix_min=4)
    gp, _, _ = plans(prob, precision=m.MM_FP64)
    with pytest.raises(m.MMError) as e:
        m.mm_autotune(gp)
    assert e.value.code == m.MM_EINVAL
