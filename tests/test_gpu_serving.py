"""Serving with continuous batching: each request's map is the same solved alone (one slot) and
in a mix that shares A-application launches, and matches the FP64 oracle (mixed-precision
tolerance: rel. map error <= 1e-5 at the same tol)."""
import time

import numpy as np
import pytest

import oracle as O
import synth
from gpu_helpers import mm

pytestmark = pytest.mark.gpu

TOL = 1e-8


def requests():
    out = []
    for i, (side, ndet, nsamp, lam) in enumerate([(64, 2, 32768, 512), (128, 4, 65536, 1024),
                                                 (96, 3, 40000, 2048)]):
        cfg = synth.tiny_config(side=side, n_det=ndet, n_samp=nsamp, lam=lam, config_id=40 + i,
                                speed=0.25 * side / 128)
        out.append(synth.to_numpy(synth.make_ground_problem(cfg)))
    return out


def submit(srv, p):
    return srv.submit(p["n_det"], p["n_int"], p["block_len"].tolist(), p["n_pix"], p["pix"], p["psi"],
                      p["lam"], p["band"], p["d"], tol=TOL)


def oracle_map(p, d=None):
    op = O.make_plan(p["pix"], p["psi"], p["block_len"], p["band"], p["n_pix"])
    x = O.pcg(op, O.rhs(op, p["d"] if d is None else d), tol=TOL, max_iter=5000).x
    m = np.zeros((p["n_pix"], 3))
    m[op.obs_to_global] = x
    return m


@pytest.fixture(scope="module")
def probs():
    return requests()


def test_alone_equals_mix_and_oracle(probs):
    m = mm()
    alone = []
    srv = m.Server(max_slots=1)
    for p in probs:
        mp, info = srv.wait(submit(srv, p))
        assert info.status == 0 and info.batch == 1 and info.true_rel_res < TOL
        alone.append(mp)
    srv.close()
    srv = m.Server(max_slots=8)
    ids = [submit(srv, p) for p in probs]
    mixed = [srv.wait(i) for i in ids]
    srv.close()
    assert max(info.batch for _, info in mixed) >= 2          # A-applies shared a launch
    for p, a, (mx, info) in zip(probs, alone, mixed):
        assert info.status == 0 and info.true_rel_res < TOL
        assert np.linalg.norm(mx - a) <= 1e-6 * np.linalg.norm(a)
        ref = oracle_map(p)
        assert np.linalg.norm(mx - ref) <= 1e-5 * np.linalg.norm(ref)


def test_request_admitted_while_another_runs(probs):
    # the long request runs a fixed 3000 iterations (unreachable tolerance), far longer than the
    # 50 ms after which the short one arrives, so the two always share launches
    m = mm()
    srv = m.Server(max_slots=4)
    p = probs[1]
    long_rid = srv.submit(p["n_det"], p["n_int"], p["block_len"].tolist(), p["n_pix"], p["pix"], p["psi"],
                          p["lam"], p["band"], p["d"], tol=1e-30, max_iter=3000)
    time.sleep(0.05)
    small = submit(srv, probs[0])
    ms, i_small = srv.wait(small)
    mb, i_long = srv.wait(long_rid, raise_on_error=False)
    srv.close()
    assert i_small.status == 0 and i_small.true_rel_res < TOL
    assert i_long.status == m.MM_ENOTCONV and i_long.iters == 3000
    assert i_small.batch >= 2 and i_long.batch >= 2           # they ran side by side


def test_admission_respects_budget_and_bad_request(probs):
    m = mm()
    srv = m.Server(hbm_budget=1, max_slots=8)                 # one request at a time
    ids = [submit(srv, p) for p in probs]
    infos = [srv.wait(i)[1] for i in ids]
    assert all(i.status == 0 and i.batch == 1 for i in infos)
    p = dict(probs[0])
    p["pix"] = p["pix"].copy()
    p["pix"][3] = p["n_pix"] + 5                              # invalid pixel: fails at admission
    bad = submit(srv, p)
    with pytest.raises(m.MMError) as e:
        srv.wait(bad)
    assert e.value.code == m.MM_EINVAL
    srv.close()


def test_fp32_tod_and_fp64_class_requests_in_one_mix(probs):
    """FP32 TOD is accepted (d_is_fp32), and FP64-class requests (double-float and IEEE FP64
    operators in every iteration) are served next to a mixed-precision one: each matches the
    oracle's PCG at the same tol, within the FP64 tolerance for the FP64-class requests."""
    m = mm()
    p = probs[1]
    args = (p["n_det"], p["n_int"], p["block_len"].tolist(), p["n_pix"], p["pix"], p["psi"], p["lam"],
            p["band"])
    d32 = p["d"].astype(np.float32)
    srv = m.Server(max_slots=8)
    r32 = srv.submit(*args, d32, tol=TOL)
    rdf = srv.submit(*args, p["d"], tol=TOL, precision=m.MM_FP64, plan_precision=m.MM_DF64)
    r64 = srv.submit(*args, p["d"], tol=TOL, precision=m.MM_FP64, plan_precision=m.MM_FP64)
    m32, i32 = srv.wait(r32)
    mdf, idf = srv.wait(rdf)
    m64, i64 = srv.wait(r64)
    srv.close()
    ref = oracle_map(p)
    ref32 = oracle_map(p, d32.astype(np.float64))
    assert i32.status == 0 and i32.true_rel_res < TOL and i32.n_apply32 > 0
    assert np.linalg.norm(m32 - ref32) <= 1e-5 * np.linalg.norm(ref32)
    for mp, info in ((mdf, idf), (m64, i64)):
        assert info.status == 0 and info.true_rel_res < TOL
        assert info.n_apply32 == 0 and info.n_apply64 >= info.iters   # FP64-class in every iteration
        assert np.linalg.norm(mp - ref) <= 1e-6 * np.linalg.norm(ref)


def test_many_concurrent_requests(probs):
    """Twenty-four requests submitted at once (16 slots, so up to 16 planned and iterated side by
    side while four planner threads build the next ones on their own streams): every one finishes
    with status 0 and the same map as the same request solved alone."""
    m = mm()
    srv = m.Server(max_slots=1)
    alone = [srv.wait(submit(srv, p))[0] for p in probs]
    srv.close()
    srv = m.Server(max_slots=16)
    order = [k % len(probs) for k in range(24)]
    ids = [submit(srv, probs[k]) for k in order]
    out = [srv.wait(i, raise_on_error=False) for i in ids]
    srv.close()
    assert max(info.batch for _, info in out) >= 8
    for k, (mp, info) in zip(order, out):
        assert info.status == 0 and info.true_rel_res < TOL
        assert np.linalg.norm(mp - alone[k]) <= 1e-6 * np.linalg.norm(alone[k])
