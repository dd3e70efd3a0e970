"""Serving engine: per-query results against the FP64 oracle, each result the same alone and in a
mixed batch, and the host-side failure paths (queue full, never-admittable query, unknown ticket),
all without any device fault."""
import time

import numpy as np
import pytest
import torch

from oracle import relnn_oracle as O
from paper_2605_24207_b300 import relnn as R
from paper_2605_24207_b300 import workloads as W

from rule_cases import OBr, bf16_round, rel_frob

pytestmark = pytest.mark.gpu


def _shared_linear(seed=0, d=64, d_out=64):
    rng = np.random.default_rng(seed)
    Wt = (rng.standard_normal((d_out, 2 * d)) / np.sqrt(2 * d)).astype(np.float32)
    b = (rng.standard_normal(d_out) / np.sqrt(2 * d)).astype(np.float32)
    return Wt, b


def _queries(sizes, seed=0, d=64):
    qs = []
    for i, n in enumerate(sizes):
        keys, src, dst, z = W.serving_query(seed, i, n, d)
        qs.append(dict(h=keys, src=src, dst=dst, z=z))
    return qs


def _dev(q):
    return (torch.from_numpy(q["h"]).cuda(), torch.from_numpy(q["z"]).cuda().to(torch.bfloat16),
            torch.from_numpy(q["src"]).cuda(), torch.from_numpy(q["dst"]).cuda())


def _run_all(server, dqs):
    tickets = [server.submit(*dq) for dq in dqs]
    res = []
    for t in tickets:
        r = None
        deadline = time.time() + 60
        while r is None and time.time() < deadline:
            r = server.poll(t, timeout_us=200_000)
        assert r is not None, "query did not complete"
        keys, out, lat, nb = r
        res.append((keys.cpu().numpy().copy(), out.cpu().numpy().copy(), lat, nb))
        server.release(t)
    return res


def test_served_results_alone_equal_mixed_and_match_oracle(gpu):
    Wn, bn = _shared_linear()
    Wt, bt = torch.from_numpy(Wn).cuda(), torch.from_numpy(bn).cuda()
    sizes = [1000, 37_000, 2500, 150_000, 8000, 1200, 60_000, 3000, 90_000, 1500, 20_000, 4000]
    qs = _queries(sizes)
    dqs = [_dev(q) for q in qs]
    mixed = R.Server(Wt, bt, 64, flags=R.FLAG_BF16, max_batch_queries=8, max_batch_tuples=300_000, n_workers=3)
    res_mix = _run_all(mixed, dqs)
    mixed.close()
    alone = R.Server(Wt, bt, 64, flags=R.FLAG_BF16, max_batch_queries=1, n_workers=1)
    res_alone = _run_all(alone, dqs)
    alone.close()
    assert max(r[3] for r in res_mix) > 1, "no query shared a batch"
    for q, rm, ra in zip(qs, res_mix, res_alone):
        assert ra[3] == 1
        assert np.array_equal(rm[0], ra[0])
        assert rel_frob(rm[1], ra[1]) <= 1e-5  # same tuples; only tile boundaries may differ
        ok, oo, _ = O.rule_forward(q["h"], bf16_round(q["z"]), [OBr(q["src"], q["dst"], bf16_round(Wn), bn)])
        assert np.array_equal(rm[0], ok)
        assert rel_frob(rm[1], oo) <= 1e-4


def test_queue_full_and_unadmittable_query(gpu):
    Wn, bn = _shared_linear()
    Wt, bt = torch.from_numpy(Wn).cuda(), torch.from_numpy(bn).cuda()
    big = _dev(_queries([400_000], seed=1)[0])
    small = _dev(_queries([1000], seed=2)[0])
    # a budget smaller than one query: rejected on the host with ENOMEM, nothing runs
    tiny = R.Server(Wt, bt, 64, mem_budget_bytes=1 << 20, n_workers=1)
    with pytest.raises(R.RelnnError) as e:
        tiny.submit(*big)
    assert e.value.status == 2
    tiny.close()
    # queue of one: while the first query is queued or running, the next submit gets EAGAIN
    s = R.Server(Wt, bt, 64, max_queue=1, n_workers=1)
    t0 = s.submit(*big)
    saw_eagain = False
    for _ in range(20):
        try:
            t1 = s.submit(*small)
        except R.RelnnError as err:
            assert err.status == 4
            saw_eagain = True
            break
        else:
            while s.poll(t1, timeout_us=100_000) is None:
                pass
            s.release(t1)
    assert saw_eagain
    while s.poll(t0, timeout_us=100_000) is None:
        pass
    s.release(t0)
    # unknown ticket
    with pytest.raises(R.RelnnError) as e:
        s.poll(123456789)
    assert e.value.status == 1
    s.close()
