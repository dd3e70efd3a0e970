"""GPU parity of the cyclic self-join (relnn_triangle_*; the DHN triangle homomorphism of paper Sec. 5)
against the FP64 oracle: every width, f32 and bf16 rows, duplicate edges and H rows, keys outside
H, sparse int64 keys, a hub whose rows span many ranges, the backward, and the closed form of the
unit-embedding case (closed 3-walk counts = diagonal of the cubed edge-multiplicity matrix)."""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from oracle import relnn_oracle as O
from paper_2605_24207_b300 import relnn as R
from paper_2605_24207_b300 import workloads as W

from rule_cases import bf16_round, rel_frob, to_dev

pytestmark = pytest.mark.gpu


def _plan(h, src, dst):
    return R.TrianglePlan(to_dev(h), to_dev(src), to_dev(dst))


@pytest.mark.parametrize("d", [32, 64, 128, 256])
@pytest.mark.parametrize("bf16", [False, True])
def test_triangle_forward_matches_oracle(gpu, d, bf16):
    h, a, b, c, src, dst = W.graph_batch(51, 400, 20, d, dup_edges=0.05, dup_rows=0.05, missing=0.02)
    T = _plan(h, src, dst)
    dt = torch.bfloat16 if bf16 else torch.float32
    out = T.forward(to_dev(a, dt), to_dev(b, dt), to_dev(c, dt))
    torch.cuda.synchronize()
    if bf16:
        a, b, c = bf16_round(a), bf16_round(b), bf16_round(c)
    ok, oo = O.triangle_forward(h, a, b, c, src, dst)
    assert np.array_equal(T.out_keys().cpu().numpy(), ok)
    assert rel_frob(out.cpu().numpy(), oo) <= 1e-5


def test_triangle_sparse_int64_keys(gpu):
    h, a, b, c, src, dst = W.graph_batch(52, 300, 16, 64, key_dtype=np.int64)
    scale = np.int64(1) << 36  # keys spread over a wide range: the hash build side
    h, src, dst = h * scale + 7, src * scale + 7, dst * scale + 7
    T = _plan(h, src, dst)
    out = T.forward(to_dev(a), to_dev(b), to_dev(c))
    ok, oo = O.triangle_forward(h, a, b, c, src, dst)
    assert np.array_equal(T.out_keys().cpu().numpy(), ok)
    assert rel_frob(out.cpu().numpy(), oo) <= 1e-5


def test_triangle_unit_embeddings_count_closed_walks(gpu):
    """a = b = c = 1: Out[n] = (M^3)[n][n] with M the edge-multiplicity matrix (exact integers)."""
    rng = np.random.default_rng(5)
    K = 300
    h = np.arange(K, dtype=np.int32)
    src = rng.integers(0, K, size=20_000).astype(np.int32)
    dst = rng.integers(0, K, size=20_000).astype(np.int32)  # repeated edges and self-loops included
    T = _plan(h, src, dst)
    ones = torch.ones((K, 32), dtype=torch.float32, device="cuda")
    out = T.forward(ones, ones, ones)
    M = sp.csr_matrix((np.ones(src.size), (src, dst)), shape=(K, K))
    diag = (M @ M @ M).diagonal()
    keys = T.out_keys().cpu().numpy()
    assert np.array_equal(keys, np.nonzero(diag)[0])
    assert np.array_equal(out.cpu().numpy()[:, 0], diag[keys].astype(np.float32))


def test_triangle_hub(gpu):
    """Node 0 points to and is pointed at by every node of a large graph: its row collects one
    record per closing node over many ranges, and its adjacency lists are long."""
    rng = np.random.default_rng(6)
    K = 4000
    h = np.arange(K, dtype=np.int32)
    ring_s = np.arange(1, K, dtype=np.int32)
    src = np.concatenate([np.zeros(K - 1, np.int32), ring_s, ring_s])
    dst = np.concatenate([ring_s, np.zeros(K - 1, np.int32), (ring_s % (K - 1)) + 1]).astype(np.int32)
    a, b, c = (rng.standard_normal((K, 64)).astype(np.float32) for _ in range(3))
    T = _plan(h, src, dst)
    out = T.forward(to_dev(a), to_dev(b), to_dev(c))
    ok, oo = O.triangle_forward(h, a, b, c, src, dst)
    assert np.array_equal(T.out_keys().cpu().numpy(), ok)
    assert rel_frob(out.cpu().numpy(), oo) <= 1e-5


@pytest.mark.parametrize("bf16", [False, True])
def test_triangle_backward(gpu, bf16):
    h, a, b, c, src, dst = W.graph_batch(53, 300, 20, 64, dup_edges=0.05, dup_rows=0.05)
    T = _plan(h, src, dst)
    dt = torch.bfloat16 if bf16 else torch.float32
    ta, tb, tc = to_dev(a, dt), to_dev(b, dt), to_dev(c, dt)
    out = T.forward(ta, tb, tc)
    dout = np.random.default_rng(7).standard_normal(tuple(out.shape)).astype(np.float32)
    da, db, dc = T.backward(to_dev(dout), ta, tb, tc)
    torch.cuda.synchronize()
    if bf16:
        a, b, c = bf16_round(a), bf16_round(b), bf16_round(c)
    oa, ob, oc = O.triangle_backward(h, a, b, c, src, dst, dout)
    assert rel_frob(da.cpu().numpy(), oa) <= 1e-5
    assert rel_frob(db.cpu().numpy(), ob) <= 1e-5
    assert rel_frob(dc.cpu().numpy(), oc) <= 1e-5


def test_triangle_without_matches_and_bad_width(gpu):
    h = np.arange(10, dtype=np.int32)
    src = np.arange(9, dtype=np.int32)
    dst = src + 1  # a path: no cycles
    T = _plan(h, src, dst)
    assert T.n_out == 0 and T.n_records == 0
    z = torch.zeros((10, 32), device="cuda")
    assert T.forward(z, z, z).shape[0] == 0
    with pytest.raises(R.RelnnError):
        T.forward(torch.zeros((10, 48), device="cuda"), torch.zeros((10, 48), device="cuda"),
                  torch.zeros((10, 48), device="cuda"))


@pytest.mark.parametrize("bf16", [False, True])
@pytest.mark.parametrize("d", [32, 128])
def test_triangle_unique_keys_read_rows_in_place(gpu, bf16, d):
    """Unique H keys: the records name H rows and the walk reads a, b, c (f32 or bf16) in place;
    forward and backward against the oracle."""
    h, a, b, c, src, dst = W.graph_batch(54, 300, 20, d, dup_edges=0.05, missing=0.02)
    T = _plan(h, src, dst)
    dt = torch.bfloat16 if bf16 else torch.float32
    ta, tb, tc = to_dev(a, dt), to_dev(b, dt), to_dev(c, dt)
    out = T.forward(ta, tb, tc)
    dout = np.random.default_rng(8).standard_normal(tuple(out.shape)).astype(np.float32)
    da, db, dc = T.backward(to_dev(dout), ta, tb, tc)
    torch.cuda.synchronize()
    if bf16:
        a, b, c = bf16_round(a), bf16_round(b), bf16_round(c)
    ok, oo = O.triangle_forward(h, a, b, c, src, dst)
    assert np.array_equal(T.out_keys().cpu().numpy(), ok)
    assert rel_frob(out.cpu().numpy(), oo) <= 1e-5
    oa, ob, oc = O.triangle_backward(h, a, b, c, src, dst, dout)
    assert rel_frob(da.cpu().numpy(), oa) <= 1e-5
    assert rel_frob(db.cpu().numpy(), ob) <= 1e-5
    assert rel_frob(dc.cpu().numpy(), oc) <= 1e-5
