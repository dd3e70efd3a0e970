"""GPU parity of streaming a relation from host memory in chunks (relnn_stream_*; paper Sec. 6 names
streaming mini-batches to the GPU as its memory-scaling direction) against the FP64 oracle on the
whole relation, and against the in-memory plan: several chunks with a ragged last one, both
forms, with a per-tuple embedding r, MEAN, a selection, pinned and pageable host memory, the
backward (dW, db, dz on the device, dr back in host memory) and the edge cases."""
import numpy as np
import pytest
import torch

from oracle import relnn_oracle as O
from paper_2605_24207_b300 import relnn as R
from paper_2605_24207_b300 import workloads as W

from rule_cases import OBr, bf16_round, oracle_rule, rel_frob, to_dev

pytestmark = pytest.mark.gpu


def _stream(rel, flags=0, chunk=7000, pin=False, filters=None, budget=0):
    br = rel.branches[0]
    src, dst = torch.from_numpy(br.src), torch.from_numpy(br.dst)
    if pin:
        src, dst = src.pin_memory(), dst.pin_memory()
    d_r = 0 if br.r is None else br.r.shape[1]
    identity = br.W is None
    if identity:
        flags |= R.FLAG_IDENTITY
    act = R.ACT_RELU if rel.act == "relu" else R.ACT_NONE
    d_out = 0 if identity else br.W.shape[0]
    return R.StreamRule(to_dev(rel.h_ids), src, dst, rel.z.shape[1], d_out, act=act, flags=flags, d_r=d_r,
                        chunk_tuples=chunk, mem_budget=budget, filters=filters)


def _inputs(rel, bf16, pin=False):
    br = rel.branches[0]
    dt = torch.bfloat16 if bf16 else torch.float32
    z = to_dev(rel.z, dt)
    Wt = None if br.W is None else to_dev(br.W, dt)
    bt = None if br.b is None else to_dev(br.b)
    r = None
    if br.r is not None:
        r = torch.from_numpy(np.ascontiguousarray(br.r, np.float32)).to(dt)
        if pin:
            r = r.pin_memory()
    return z, Wt, bt, r


@pytest.mark.parametrize("bf16", [False, True])
@pytest.mark.parametrize("act", ["none", "relu"])
def test_stream_forward_matches_oracle(gpu, bf16, act):
    d = 64 if bf16 else 16
    rel = W.make_rule(81, 40_000, 3000, d, 32 if bf16 else 24, np.int32, act=act, d_r=16 if bf16 else 8,
                      src_dist="zipf", src_s=1.2, missing_frac=0.02)
    S = _stream(rel, flags=R.FLAG_BF16 if bf16 else 0, chunk=7000, pin=bf16)
    assert S.n_chunks == 6 and S.chunk_tuples == 7000
    z, Wt, bt, r = _inputs(rel, bf16, pin=bf16)
    keys, out = S.forward(z, Wt, bt, r)
    torch.cuda.synchronize()
    ok, oo, _ = oracle_rule(rel, round_z=bf16, round_r=bf16, round_w=bf16)
    assert np.array_equal(keys.cpu().numpy(), ok)
    assert rel_frob(out.cpu().numpy(), oo) <= (1e-4 if bf16 else 1e-5)


def test_stream_equals_the_in_memory_plan(gpu):
    """Same relation, one device-resident plan against six streamed chunks: same key set and the
    same values up to the order of f32 additions across chunks."""
    rel = W.make_rule(82, 50_000, 4000, 64, 64, np.int64, src_dist="zipf", src_s=1.1, sparse_keys=True)
    br = rel.branches[0]
    z, Wt, bt, _ = _inputs(rel, True)
    plan = R.RulePlan(to_dev(rel.h_ids), [(to_dev(br.src), to_dev(br.dst))], 64, 64, flags=R.FLAG_BF16)
    ref = plan.forward(z, [Wt], [bt])
    S = _stream(rel, flags=R.FLAG_BF16, chunk=9000)
    keys, out = S.forward(z, Wt, bt)
    torch.cuda.synchronize()
    assert torch.equal(keys, plan.out_keys())
    assert rel_frob(out.cpu().numpy(), ref.cpu().numpy().astype(np.float64)) <= 1e-6


@pytest.mark.parametrize("bf16", [False, True])
def test_stream_backward_matches_oracle(gpu, bf16):
    d = 64 if bf16 else 16
    rel = W.make_rule(83, 30_000, 2500, d, 32, np.int32, act="relu", d_r=16 if bf16 else 8, dst_dist="zipf",
                      dst_s=1.2)
    S = _stream(rel, flags=R.FLAG_BF16 if bf16 else 0, chunk=8000)
    z, Wt, bt, r = _inputs(rel, bf16)
    keys, out = S.forward(z, Wt, bt, r)
    dout = np.random.default_rng(8).standard_normal(tuple(out.shape)).astype(np.float32)
    dW, db, dz, dr = S.backward(to_dev(dout), z, Wt, bt, r)
    torch.cuda.synchronize()
    br = rel.branches[0]
    rd = (lambda a: bf16_round(a)) if bf16 else (lambda a: a)
    o = OBr(br.src, br.dst, rd(br.W), br.b, rd(br.r))
    oW, ob, oz, orr = O.rule_backward(rel.h_ids, rd(rel.z), [o], keys.cpu().numpy(), dout, act="relu")
    tol = 2e-2 if bf16 else 1e-5
    assert rel_frob(dW.cpu().numpy(), oW[0]) <= tol
    assert rel_frob(db.cpu().numpy(), ob[0]) <= 1e-5
    assert rel_frob(dz.cpu().numpy(), oz) <= tol
    assert rel_frob(dr.numpy(), orr[0]) <= tol


def test_stream_mean_with_selection(gpu):
    rel = W.make_rule(84, 30_000, 2000, 16, 16, np.int32, act="relu")
    flt = [("src", "<", "dst"), ("dst", "!=", 5)]
    S = _stream(rel, flags=R.FLAG_MEAN, chunk=6000, filters=flt)
    z, Wt, bt, _ = _inputs(rel, False)
    keys, out = S.forward(z, Wt, bt)
    br = rel.branches[0]
    o = OBr(br.src, br.dst, br.W, br.b, None, flt)
    ok, oo, _ = O.rule_forward(rel.h_ids, rel.z, [o], act="relu", agg="mean")
    assert np.array_equal(keys.cpu().numpy(), ok)
    assert rel_frob(out.cpu().numpy(), oo) <= 1e-5
    dout = np.random.default_rng(3).standard_normal(tuple(out.shape)).astype(np.float32)
    dW, db, dz, _ = S.backward(to_dev(dout), z, Wt, bt)
    oW, ob, oz, _ = O.rule_backward(rel.h_ids, rel.z, [o], ok, dout, act="relu", agg="mean")
    assert rel_frob(dW.cpu().numpy(), oW[0]) <= 1e-5
    assert rel_frob(db.cpu().numpy(), ob[0]) <= 1e-5
    assert rel_frob(dz.cpu().numpy(), oz) <= 1e-5


def test_stream_chunk_from_the_memory_budget(gpu):
    """chunk_tuples = 0: the chunk size follows the device-memory budget (several chunks here)."""
    rel = W.make_rule(85, 60_000, 3000, 16, 16, np.int32)
    S = _stream(rel, chunk=0, budget=4 << 20)
    assert S.n_chunks >= 2
    z, Wt, bt, _ = _inputs(rel, False)
    keys, out = S.forward(z, Wt, bt)
    ok, oo, _ = oracle_rule(rel)
    assert np.array_equal(keys.cpu().numpy(), ok)
    assert rel_frob(out.cpu().numpy(), oo) <= 1e-5


def test_stream_single_chunk_and_empty(gpu):
    rel = W.make_rule(86, 5000, 800, 16, 16, np.int32)
    S = _stream(rel, chunk=1 << 20)
    assert S.n_chunks == 1
    z, Wt, bt, _ = _inputs(rel, False)
    keys, out = S.forward(z, Wt, bt)
    ok, oo, _ = oracle_rule(rel)
    assert np.array_equal(keys.cpu().numpy(), ok) and rel_frob(out.cpu().numpy(), oo) <= 1e-5
    empty = W.make_rule(87, 0, 300, 16, 16, np.int32)
    S0 = _stream(empty, chunk=1000)
    assert S0.n_chunks == 0
    keys, out = S0.forward(*_inputs(empty, False)[:3])
    assert keys.numel() == 0 and out.shape[0] == 0


def test_stream_rejects_unsupported_flags(gpu):
    rel = W.make_rule(88, 2000, 300, 16, 16, np.int32)
    for f in (R.FLAG_MAX, R.FLAG_PUSHDOWN | R.FLAG_BF16, R.FLAG_NO_JOIN_DST):
        with pytest.raises(R.RelnnError):
            _stream(rel, flags=f)
    S = _stream(rel)
    z, Wt, bt, _ = _inputs(rel, False)
    with pytest.raises(R.RelnnError):  # the backward needs a forward's output rows
        S.backward(torch.zeros((1, 16), device="cuda"), z, Wt, bt)
