"""The failure paths that a run on a healthy device can reach without faulting or hanging it:

- a bounded wait that runs out: one CTA waits, with the library's bounded mbarrier wait, on a barrier
  nothing arrives at under a budget of a few milliseconds; the kernel must return, the call must
  report RELNN_EDEVICE / RELNN_DEV_TIMEOUT, and a rule evaluated right after must still match the
  FP64 oracle (the context stays usable);
- a serving poll that runs out: a query of a million tuples polled 50 microseconds after submission
  reports RELNN_ETIMEDOUT, and the same ticket completes afterwards."""
import ctypes as C
import time

import numpy as np
import pytest
import torch

from paper_2605_24207_b300 import relnn as R
from paper_2605_24207_b300 import workloads as W

from rule_cases import oracle_rule, rel_frob, run_rule

pytestmark = pytest.mark.gpu

EDEVICE, ETIMEDOUT, DEV_TIMEOUT = 7, 5, 1


def test_bounded_wait_times_out_and_device_stays_usable(gpu):
    L = R.lib()
    t0 = time.perf_counter()
    st = L.relnn_test_wait_timeout(3000, None)
    dt = time.perf_counter() - t0
    assert st == EDEVICE
    assert L.relnn_last_device_error() == DEV_TIMEOUT
    assert 0.003 <= dt < 1.0
    rel = W.make_rule(201, 5000, 400, 64, 64, np.int32)
    keys, out, plan, _ = run_rule(rel, flags=R.FLAG_BF16, z_dtype=torch.bfloat16)
    ok, oo, _ = oracle_rule(rel, round_z=True, round_w=True)
    assert np.array_equal(keys, ok)
    assert rel_frob(out, oo) <= 1e-4


def test_serve_poll_times_out_then_completes(gpu):
    rng = np.random.default_rng(3)
    Wt = torch.from_numpy((rng.standard_normal((64, 128)) / np.sqrt(128)).astype(np.float32)).cuda()
    bt = torch.from_numpy((rng.standard_normal(64) / np.sqrt(128)).astype(np.float32)).cuda()
    srv = R.Server(Wt, bt, 64, flags=R.FLAG_BF16, n_workers=1)
    try:
        keys, src, dst, z = W.serving_query(5, 1_000_000, 1_000_000, 64)
        q = (torch.from_numpy(keys).cuda(), torch.from_numpy(z).cuda().to(torch.bfloat16),
             torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda())
        # twelve 1M-tuple queries on one worker: the last one completes milliseconds after submission,
        # far beyond the 50 us poll (whose wait may oversleep by the OS timer slack)
        tickets = [srv.submit(*q) for _ in range(12)]
        res = R.Result()
        st = srv.L.relnn_serve_poll(srv._h, tickets[-1], C.byref(res), 50)
        assert st == ETIMEDOUT
        for t in tickets:
            r = None
            for _ in range(200):
                r = srv.poll(t, 100_000)
                if r is not None:
                    break
            assert r is not None and r[0].numel() > 0
            srv.release(t)
    finally:
        srv.close()
