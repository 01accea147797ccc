"""The serving workload's arrival process (bench.py): submissions follow an absolute Poisson
schedule, submission i at t0 + gap_0 + ... + gap_i, so a slow submission (a client copying a large
request) does not stretch the gaps that follow it and thin the offered stream.  Checked on the CPU
with a stand-in server whose submit takes 30 ms against 50 ms mean gaps."""
import os
import sys
import time
from types import SimpleNamespace

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class FakeServer:
    submit_s = 0.03

    def __init__(self, max_slots=16):
        self.t_submit = []

    def submit(self, *args, **kw):
        self.t_submit.append(time.perf_counter())
        time.sleep(self.submit_s)
        return len(self.t_submit)

    def wait(self, rid, raise_on_error=True):
        return None, SimpleNamespace(t_queue_ms=1.0, t_ms=2.0)

    def close(self):
        pass


def test_submissions_keep_the_absolute_schedule():
    servers = []

    def make(max_slots=16):
        servers.append(FakeServer(max_slots))
        return servers[-1]

    fake_mm = SimpleNamespace(Server=make, MM_FP64=1, MM_DF64=2)
    pool = [{"n_det": 1, "n_int": 1, "block_len": np.array([4]), "n_pix": 1, "pix": None, "psi": None,
             "lam": 0, "band": None, "d": None}]
    rng = np.random.default_rng(0)
    gaps = rng.exponential(0.05, size=12)
    order = np.zeros(12, dtype=int)
    lat, infos, dt, sub = bench._serve(fake_mm, pool, order, gaps, fp64=False)
    srv = servers[0]
    t = np.array(srv.t_submit[1:])          # the first submission is the warm-up
    t0 = t[0] - gaps[0]
    due = t0 + np.cumsum(gaps)
    lag = t - due
    # a submission starts at its arrival time, or right after the previous one when that ran late
    assert np.all(lag > -2e-3)
    late = np.maximum(0.0, (t[:-1] + FakeServer.submit_s) - due[1:])
    assert np.all(lag[1:] <= late + 0.05)
    # the whole stream takes about the sum of the gaps (plus the last submission), not the sum of
    # the gaps and all twelve submissions (0.36 s more)
    assert dt < gaps.sum() + 0.2
    assert len(lat) == 12 and abs(sub[0] - 1e3 * FakeServer.submit_s) < 15
