"""Pins for the FP64 oracle against things other than itself (CPU only).

Each check is chosen so that a plausible slip in the oracle (a dropped term, a swapped operand, a
wrong index, set instead of bag semantics) fails at least one of them:
  * nested-loop brute force over E x H x H (join, Linear, SUM written as explicit loops);
  * the join cardinality identity |E |><| H |><| H| = sum_e cnt_H(src_e) * cnt_H(dst_e);
  * closed forms: W = [I;0], b = 0 equals a sparse incidence product (scipy); W = [0;I] gives
    deg(k) z_k; W = 0 gives deg(k) b;
  * union = sum of branches; invariance under row permutations of E and H; linearity in (W, b);
  * a hand-derived golden example (tests/golden/hand_rule.json);
  * central finite differences (h = 1e-3) and the adjoint identity for the backward.
"""
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import relnn_oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden", "hand_rule.json")


class Br:
    def __init__(self, src, dst, W, b, r=None):
        self.src, self.dst, self.W, self.b, self.r = src, dst, W, b, r


def tiny(seed, n_e=40, n_h=12, d=3, d_out=4, d_r=0, key_range=10, key_dtype=np.int64, neg=False):
    """Tiny relations with duplicate H keys, keys missing from H and (optionally) negative keys."""
    rng = np.random.default_rng(seed)
    lo = -key_range if neg else 0
    h_ids = rng.integers(lo, key_range, size=n_h).astype(key_dtype)
    z = rng.standard_normal((n_h, d))
    src = rng.integers(lo, key_range + 3, size=n_e).astype(key_dtype)
    dst = rng.integers(lo, key_range + 3, size=n_e).astype(key_dtype)
    d_in = 2 * d + d_r
    W = rng.standard_normal((d_out, d_in))
    b = rng.standard_normal(d_out)
    r = rng.standard_normal((n_e, d_r)) if d_r else None
    return h_ids, z, Br(src, dst, W, b, r)


# ----------------------------------------------------------------------------- brute force
def brute_join(src, dst, h_ids, join_dst=True):
    out = []
    for e in range(len(src)):
        for a in range(len(h_ids)):
            if h_ids[a] != src[e]:
                continue
            if not join_dst:
                out.append((e, a, -1))
                continue
            for c in range(len(h_ids)):
                if h_ids[c] == dst[e]:
                    out.append((e, a, c))
    return sorted(out)


def brute_rule(h_ids, z, branches, act="none", join_dst=True, concat_dst=True):
    acc = {}
    for br in branches:
        for (e, a, c) in brute_join(br.src, br.dst, h_ids, join_dst):
            x = list(z[a])
            if concat_dst:
                x += list(z[c])
            if br.r is not None:
                x += list(br.r[e])
            if br.W is None:
                y = x
            else:
                y = []
                for o in range(len(br.W)):
                    s = br.b[o]
                    for k in range(len(x)):
                        s += br.W[o][k] * x[k]
                    y.append(s)
            if act == "relu":
                y = [v if v > 0 else 0.0 for v in y]
            key = br.dst[e]
            if key not in acc:
                acc[key] = [0.0] * len(y)
            acc[key] = [p + q for p, q in zip(acc[key], y)]
    keys = sorted(acc)
    return keys, np.array([acc[k] for k in keys])


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("join_dst", [True, False])
def test_join_matches_nested_loops(seed, join_dst):
    h_ids, z, br = tiny(seed, neg=(seed % 2 == 1), key_dtype=np.int32 if seed % 3 == 0 else np.int64)
    e, hs, hd = O.join(br.src, br.dst, h_ids, join_dst)
    got = sorted(zip(e.tolist(), hs.tolist(), hd.tolist()))
    assert got == brute_join(br.src.tolist(), br.dst.tolist(), h_ids.tolist(), join_dst)
    # the oracle's own order is already (e, hs, hd) ascending
    assert list(zip(e.tolist(), hs.tolist(), hd.tolist())) == got


@pytest.mark.parametrize("seed", range(6))
def test_join_cardinality_identity(seed):
    h_ids, z, br = tiny(seed, n_e=64, n_h=20, key_range=6)
    e, _, _ = O.join(br.src, br.dst, h_ids)
    cnt = {}
    for k in h_ids.tolist():
        cnt[k] = cnt.get(k, 0) + 1
    expect = sum(cnt.get(s, 0) * cnt.get(d, 0) for s, d in zip(br.src.tolist(), br.dst.tolist()))
    assert e.size == expect == O.join_cardinality(br.src, br.dst, h_ids)
    # one-sided form: sum over keys of c_probe(k) * c_build(k)
    pr, bu = O.join_pairs(br.src, h_ids)
    cp = {}
    for k in br.src.tolist():
        cp[k] = cp.get(k, 0) + 1
    assert pr.size == sum(c * cnt.get(k, 0) for k, c in cp.items())
    assert sorted(zip(pr.tolist(), bu.tolist())) == sorted(
        (i, j) for i in range(br.src.size) for j in range(h_ids.size) if br.src[i] == h_ids[j])


@pytest.mark.parametrize("seed", range(5))
@pytest.mark.parametrize("act", ["none", "relu"])
def test_forward_matches_brute_force(seed, act):
    h_ids, z, br = tiny(seed, d_r=2 if seed % 2 else 0)
    keys, out, sizes = O.rule_forward(h_ids, z, [br], act=act)
    bk, bo = brute_rule(h_ids, z, [br], act=act)
    assert keys.tolist() == bk
    np.testing.assert_allclose(out, bo, rtol=1e-12, atol=1e-12)
    assert sizes[0] == len(brute_join(br.src, br.dst, h_ids))


def test_forward_readout_form_matches_brute_force():
    h_ids, z, br = tiny(7)
    br.W, br.b = None, None
    keys, out, _ = O.rule_forward(h_ids, z, [br], join_dst=False, concat_dst=False)
    bk, bo = brute_rule(h_ids, z, [br], join_dst=False, concat_dst=False)
    assert keys.tolist() == bk
    np.testing.assert_allclose(out, bo, rtol=1e-12, atol=1e-12)


def test_union_matches_brute_force_and_is_sum_of_branches():
    h_ids, z, b1 = tiny(11, d_r=2)
    _, _, b2 = tiny(12, d_r=2)
    _, _, b3 = tiny(13, d_r=2)
    b2.W = np.random.default_rng(5).standard_normal(b1.W.shape)
    keys, out, _ = O.rule_forward(h_ids, z, [b1, b2, b3])
    bk, bo = brute_rule(h_ids, z, [b1, b2, b3])
    assert keys.tolist() == bk
    np.testing.assert_allclose(out, bo, rtol=1e-12, atol=1e-12)
    acc = {}
    for br in (b1, b2, b3):
        k, o, _ = O.rule_forward(h_ids, z, [br])
        for kk, row in zip(k.tolist(), o):
            acc[kk] = acc.get(kk, 0) + row
    np.testing.assert_allclose(out, np.array([acc[k] for k in keys.tolist()]), rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("seed", range(4))
def test_identity_linear_is_sparse_incidence_product(seed):
    """W = [I; 0], b = 0: H'[k] = sum over matched tuples with dst = k of z[hs] = A^T Z, where A is
    the (tuple x H-row) incidence of the src side restricted to tuples whose dst matches."""
    h_ids, z, br = tiny(seed, n_e=80, n_h=15, d=3, d_out=3, key_range=8)
    d = z.shape[1]
    br.W = np.concatenate([np.eye(d), np.zeros((d, d))], axis=1)
    br.b = np.zeros(d)
    keys, out, _ = O.rule_forward(h_ids, z, [br])
    # independent construction with scipy.sparse: rows = distinct output keys, cols = H rows
    cnt = {}
    for k in h_ids.tolist():
        cnt[k] = cnt.get(k, 0) + 1
    uk = sorted({dd for s, dd in zip(br.src.tolist(), br.dst.tolist()) if s in cnt and dd in cnt})
    rowpos = {k: i for i, k in enumerate(uk)}
    rr, cc = [], []
    for s, dd in zip(br.src.tolist(), br.dst.tolist()):
        if s in cnt and dd in cnt:
            for j in range(h_ids.size):
                if h_ids[j] == s:
                    for _ in range(cnt[dd]):
                        rr.append(rowpos[dd])
                        cc.append(j)
    A = sp.coo_matrix((np.ones(len(rr)), (rr, cc)), shape=(len(uk), h_ids.size)).tocsr()
    assert keys.tolist() == uk
    np.testing.assert_allclose(out, A @ z, rtol=1e-12, atol=1e-12)


def _deg(br, h_ids, keys):
    cnt = {}
    for k in h_ids.tolist():
        cnt[k] = cnt.get(k, 0) + 1
    deg = {}
    for s, d in zip(br.src.tolist(), br.dst.tolist()):
        m = cnt.get(s, 0) * cnt.get(d, 0)
        if m:
            deg[d] = deg.get(d, 0) + m
    return np.array([deg[k] for k in keys.tolist()], np.float64)


def test_closed_forms_dst_identity_and_zero_weight():
    h_ids, z, br = tiny(3, n_e=60, n_h=10, key_range=12)
    # unique H keys so that z_dst is the embedding of the key itself
    h_ids = np.arange(10, dtype=np.int64) * 3 - 7
    br.src = h_ids[np.random.default_rng(1).integers(0, 10, 60)]
    br.dst = h_ids[np.random.default_rng(2).integers(0, 10, 60)]
    d = z.shape[1]
    br.W = np.concatenate([np.zeros((d, d)), np.eye(d)], axis=1)
    br.b = np.zeros(d)
    keys, out, _ = O.rule_forward(h_ids, z, [br])
    deg = _deg(br, h_ids, keys)
    zk = np.array([z[h_ids.tolist().index(k)] for k in keys.tolist()])
    np.testing.assert_allclose(out, deg[:, None] * zk, rtol=1e-12, atol=1e-12)
    br.W = np.zeros((4, 2 * d))
    br.b = np.array([1.0, -2.0, 0.5, 3.0])
    keys, out, _ = O.rule_forward(h_ids, z, [br])
    np.testing.assert_allclose(out, _deg(br, h_ids, keys)[:, None] * br.b[None, :], rtol=1e-12)


def test_permutation_invariance():
    h_ids, z, br = tiny(21, n_e=70, d_r=2)
    keys, out, _ = O.rule_forward(h_ids, z, [br])
    rng = np.random.default_rng(0)
    pe = rng.permutation(br.src.size)
    ph = rng.permutation(h_ids.size)
    br2 = Br(br.src[pe], br.dst[pe], br.W, br.b, br.r[pe])
    k2, o2, _ = O.rule_forward(h_ids[ph], z[ph], [br2])
    assert k2.tolist() == keys.tolist()
    np.testing.assert_allclose(o2, out, rtol=1e-11, atol=1e-11)


def test_linearity_in_weights():
    h_ids, z, br = tiny(22, n_e=50)
    rng = np.random.default_rng(3)
    W2, b2 = rng.standard_normal(br.W.shape), rng.standard_normal(br.b.shape)
    a, c = 0.7, -1.3
    k1, o1, _ = O.rule_forward(h_ids, z, [br])
    _, o2, _ = O.rule_forward(h_ids, z, [Br(br.src, br.dst, W2, b2)])
    _, o3, _ = O.rule_forward(h_ids, z, [Br(br.src, br.dst, a * br.W + c * W2, a * br.b + c * b2)])
    np.testing.assert_allclose(o3, a * o1 + c * o2, rtol=1e-11, atol=1e-11)


# ----------------------------------------------------------------------------- golden
def test_golden_hand_example():
    g = json.load(open(GOLD))
    h = np.array(g["h_ids"], np.int64)
    z = np.array(g["z"], np.float64)
    br = Br(np.array(g["src"]), np.array(g["dst"]), np.array(g["W"], float), np.array(g["b"], float))
    e, hs, hd = O.join(br.src, br.dst, h)
    assert [list(t) for t in zip(e.tolist(), hs.tolist(), hd.tolist())] == g["triples"]
    keys, out, _ = O.rule_forward(h, z, [br])
    assert keys.tolist() == g["out_keys"]
    assert out.tolist() == g["out"]
    _, out_r, _ = O.rule_forward(h, z, [br], act="relu")
    assert out_r.tolist() == g["out_relu"]
    br2 = Br(np.array(g["src2"]), np.array(g["dst2"]), np.array(g["W2"], float), np.array(g["b2"], float))
    _, out_u, _ = O.rule_forward(h, z, [br, br2])
    assert out_u.tolist() == g["out_union"]
    dW, db, dz, _ = O.rule_backward(h, z, [br], keys, np.ones_like(out))
    assert dW[0].tolist() == g["dW_ones"]
    assert db[0].tolist() == g["db_ones"]
    assert dz.tolist() == g["dz_ones"]


# ----------------------------------------------------------------------------- backward
def _loss(h_ids, z, brs, act, C):
    keys, out, _ = O.rule_forward(h_ids, z, brs, act=act)
    return float(np.sum(C[: out.shape[0]] * out)), keys, out


@pytest.mark.parametrize("act", ["none", "relu"])
def test_backward_finite_differences(act):
    h_ids, z, br = tiny(31, n_e=30, n_h=10, d=3, d_out=4, d_r=2)
    keys, out, _ = O.rule_forward(h_ids, z, [br], act=act)
    C = np.random.default_rng(4).standard_normal(out.shape)
    if act == "relu":
        # keep every pre-activation away from the kink so that h = 1e-3 stays on one side
        e, hs, hd = O.join(br.src, br.dst, h_ids)
        pre = O.concat_rows(z, br.r, e, hs, hd) @ br.W.T + br.b
        assert np.min(np.abs(pre)) > 1e-2
    dW, db, dz, dr = O.rule_backward(h_ids, z, [br], keys, C, act=act)
    h = 1e-3
    rng = np.random.default_rng(9)

    def fd(arr, idx, setter):
        old = arr[idx]
        arr[idx] = old + h
        lp = _loss(h_ids, z, [br], act, C)[0]
        arr[idx] = old - h
        lm = _loss(h_ids, z, [br], act, C)[0]
        arr[idx] = old
        return (lp - lm) / (2 * h)

    for _ in range(6):
        i = tuple(rng.integers(0, s) for s in br.W.shape)
        assert fd(br.W, i, None) == pytest.approx(dW[0][i], rel=1e-6, abs=1e-8)
        j = int(rng.integers(0, br.b.size))
        assert fd(br.b, j, None) == pytest.approx(db[0][j], rel=1e-6, abs=1e-8)
        k = tuple(rng.integers(0, s) for s in z.shape)
        assert fd(z, k, None) == pytest.approx(dz[k], rel=1e-6, abs=1e-8)
        m = tuple(rng.integers(0, s) for s in br.r.shape)
        assert fd(br.r, m, None) == pytest.approx(dr[0][m], rel=1e-6, abs=1e-8)


def test_backward_adjoint_identity():
    """<dOut, J v> = <J^T dOut, v> for the map (z, r) -> H' at fixed weights (linear when act=none)."""
    h_ids, z, br = tiny(41, n_e=40, n_h=12, d=3, d_out=5, d_r=2)
    rng = np.random.default_rng(2)
    br.b = np.zeros_like(br.b)  # pure linear map in (z, r)
    keys, out, _ = O.rule_forward(h_ids, z, [br])
    dout = rng.standard_normal(out.shape)
    vz, vr = rng.standard_normal(z.shape), rng.standard_normal(br.r.shape)
    _, Jv, _ = O.rule_forward(h_ids, vz, [Br(br.src, br.dst, br.W, br.b, vr)])
    _, _, dz, dr = O.rule_backward(h_ids, z, [br], keys, dout)
    lhs = float(np.sum(dout * Jv))
    rhs = float(np.sum(dz * vz) + np.sum(dr[0] * vr))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def _stacked_case(seed=0):
    rng = np.random.default_rng(seed)
    K, T, d = 14, 60, 4
    h_ids = rng.permutation(K).astype(np.int64) * 5
    z = rng.standard_normal((K, d))
    src = h_ids[rng.integers(0, K, T)]
    dst = h_ids[rng.integers(0, K, T)]
    W1, b1 = rng.standard_normal((d, 2 * d)) * 0.5, rng.standard_normal(d) * 0.5
    W2, b2 = rng.standard_normal((d, 2 * d)) * 0.5, rng.standard_normal(d) * 0.5
    g_groups = rng.integers(0, 3, K).astype(np.int64)
    t_groups = np.arange(3, dtype=np.int64)
    targets = rng.standard_normal((3, d))
    return h_ids, z, src, dst, W1, b1, W2, b2, h_ids.copy(), g_groups, t_groups, targets


def test_stacked_gradient_finite_differences():
    args = list(_stacked_case())
    f = O.stacked_forward(*args)
    g = O.stacked_backward(*args, fwd=f)
    h = 1e-3
    rng = np.random.default_rng(1)
    names = {1: "dz", 4: "dW1", 5: "db1", 6: "dW2", 7: "db2"}
    checked = 0
    for pos, gname in names.items():
        arr = args[pos]
        for _ in range(5):
            i = tuple(int(rng.integers(0, s)) for s in arr.shape)
            old = arr[i]
            arr[i] = old + h
            lp = O.stacked_forward(*args)["loss"]
            arr[i] = old - h
            lm = O.stacked_forward(*args)["loss"]
            arr[i] = old
            fd = (lp - lm) / (2 * h)
            assert fd == pytest.approx(g[gname][i], rel=1e-4, abs=1e-6)
            checked += 1
    assert checked == 25


def test_mse_matches_definition_and_gradient():
    pk = np.array([0, 1, 2, 5])
    p = np.arange(8.0).reshape(4, 2)
    tk = np.array([2, 0, 1])
    t = np.array([[1.0, 1.0], [0.0, 0.0], [2.0, 2.0]])
    # joined pairs: 0<->t[1], 1<->t[2], 2<->t[0]; key 5 joins nothing
    want = np.mean(np.array([[0, 1], [0, 1], [3, 4]], float) ** 2)
    assert O.mse(pk, p, tk, t) == pytest.approx(want)
    g = O.mse_grad(pk, p, tk, t)
    assert g[3].tolist() == [0.0, 0.0]
    assert g[2].tolist() == [2 * 3 / 6, 2 * 4 / 6]


# ----------------------------------------------------------------------------- planted mistakes
def test_pins_detect_planted_mistakes(monkeypatch):
    """Plant typical slips in the oracle (on the CPU) and check that a pin above catches each."""
    g = json.load(open(GOLD))
    h = np.array(g["h_ids"], np.int64)
    z = np.array(g["z"], np.float64)
    br = Br(np.array(g["src"]), np.array(g["dst"]), np.array(g["W"], float), np.array(g["b"], float))
    good = O.rule_forward(h, z, [br])[1].tolist()
    assert good == g["out"]
    orig_tau, orig_concat, orig_index = O._tau, O.concat_rows, O.key_index

    # dropped bias term
    monkeypatch.setattr(O, "_tau", lambda X, W, b, act: orig_tau(X, W, None, act))
    assert O.rule_forward(h, z, [br])[1].tolist() != g["out"]
    monkeypatch.setattr(O, "_tau", orig_tau)
    # swapped Concat order
    monkeypatch.setattr(O, "concat_rows", lambda z_, r, e, hs, hd, c=True: orig_concat(z_, r, e, hd, hs, c))
    assert O.rule_forward(h, z, [br])[1].tolist() != g["out"]
    monkeypatch.setattr(O, "concat_rows", orig_concat)
    # set semantics on H (first duplicate only)
    monkeypatch.setattr(O, "key_index", lambda ids: {k: v[:1] for k, v in orig_index(ids).items()})
    e, _, _ = O.join(br.src, br.dst, h)
    assert e.size != len(g["triples"])
    monkeypatch.setattr(O, "key_index", orig_index)


# ----------------------------------------------------------------------------- MEAN aggregator
def brute_mean(h_ids, z, br, act="none"):
    """Per-key average of the brute-force tuple outputs (explicit loops, one branch)."""
    sums, cnts = {}, {}
    for (e, a, c) in brute_join(br.src, br.dst, h_ids):
        x = list(z[a]) + list(z[c])
        y = [br.b[o] + sum(br.W[o][k] * x[k] for k in range(len(x))) for o in range(len(br.W))]
        if act == "relu":
            y = [v if v > 0 else 0.0 for v in y]
        key = br.dst[e]
        sums[key] = [p + q for p, q in zip(sums.get(key, [0.0] * len(y)), y)]
        cnts[key] = cnts.get(key, 0) + 1
    keys = sorted(sums)
    return keys, np.array([[v / cnts[k] for v in sums[k]] for k in keys])


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("act", ["none", "relu"])
def test_mean_matches_brute_force(seed, act):
    h_ids, z, br = tiny(seed + 70)
    keys, out, _ = O.rule_forward(h_ids, z, [br], act=act, agg="mean")
    bk, bo = brute_mean(h_ids, z, br, act)
    assert list(keys) == bk
    np.testing.assert_allclose(out, bo, rtol=1e-12, atol=1e-12)


def test_mean_times_count_is_sum():
    h_ids, z, br = tiny(80, n_e=60)
    keys, mean, _ = O.rule_forward(h_ids, z, [br], agg="mean")
    keys_s, total, _ = O.rule_forward(h_ids, z, [br])
    e, hs, hd = O.join(br.src, br.dst, h_ids)
    cnt = {k: c for k, c in zip(*np.unique(np.asarray(br.dst)[e], return_counts=True))}
    assert np.array_equal(keys, keys_s)
    np.testing.assert_allclose(mean * np.array([cnt[k] for k in keys])[:, None], total, rtol=1e-12, atol=1e-12)


def test_mean_backward_finite_differences():
    h_ids, z, br = tiny(81, n_e=30, n_h=10, d=3, d_out=4)
    keys, out, _ = O.rule_forward(h_ids, z, [br], agg="mean")
    C = np.random.default_rng(5).standard_normal(out.shape)
    dW, db, dz, _ = O.rule_backward(h_ids, z, [br], keys, C, agg="mean")
    h = 1e-3

    def loss():
        k2, o2, _ = O.rule_forward(h_ids, z, [br], agg="mean")
        return float(np.sum(o2 * C))

    rng = np.random.default_rng(11)
    for arr, grad in ((br.W, dW[0]), (br.b, db[0]), (z, dz)):
        for _ in range(4):
            i = tuple(rng.integers(0, s) for s in arr.shape)
            old = arr[i]
            arr[i] = old + h
            lp = loss()
            arr[i] = old - h
            lm = loss()
            arr[i] = old
            assert (lp - lm) / (2 * h) == pytest.approx(grad[i], rel=1e-6, abs=1e-8)


# ----------------------------------------------------------------------------- selection
FILTER_SETS = [[("src", "<", "dst")], [("dst", "!=", 3), ("src", ">=", 2)], [(4, ">", "src")],
               [("src", "==", "dst")]]


@pytest.mark.parametrize("filters", FILTER_SETS)
def test_selection_matches_brute_force(filters):
    h_ids, z, br = tiny(90, n_e=50)
    br.filters = filters
    ops = {"==": lambda a, b: a == b, "!=": lambda a, b: a != b, "<": lambda a, b: a < b,
           "<=": lambda a, b: a <= b, ">": lambda a, b: a > b, ">=": lambda a, b: a >= b}
    keep = []
    for e in range(len(br.src)):
        ok = True
        for lhs, op, rhs in filters:
            val = lambda x: br.src[e] if x == "src" else (br.dst[e] if x == "dst" else x)
            ok = ok and ops[op](val(lhs), val(rhs))
        keep.append(ok)
    keep = np.array(keep)
    sub = Br(br.src[keep], br.dst[keep], br.W, br.b)
    bk, bo = brute_rule(h_ids, z, [sub])
    keys, out, _ = O.rule_forward(h_ids, z, [br])
    assert list(keys) == bk
    np.testing.assert_allclose(out, bo, rtol=1e-12, atol=1e-12)


def test_selection_is_the_rule_over_the_kept_rows():
    h_ids, z, br = tiny(91, n_e=60, d_r=2)
    br.filters = [("src", "<=", "dst"), ("dst", ">", 1)]
    keep = O.selected_rows(br)
    sub = Br(br.src[keep], br.dst[keep], br.W, br.b, br.r[keep])
    k1, o1, s1 = O.rule_forward(h_ids, z, [br])
    k2, o2, s2 = O.rule_forward(h_ids, z, [sub])
    assert np.array_equal(k1, k2) and s1 == s2
    np.testing.assert_allclose(o1, o2, rtol=1e-12, atol=1e-12)
    C = np.random.default_rng(7).standard_normal(o1.shape)
    g1 = O.rule_backward(h_ids, z, [br], k1, C)
    g2 = O.rule_backward(h_ids, z, [sub], k2, C)
    np.testing.assert_allclose(g1[0][0], g2[0][0], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(g1[2], g2[2], rtol=1e-12, atol=1e-12)
    # dr keeps the full E shape: rows that fail the selection get no gradient
    assert np.all(g1[3][0][~keep] == 0)
    np.testing.assert_allclose(g1[3][0][keep], g2[3][0], rtol=1e-12, atol=1e-12)


# ----------------------------------------------------------------------------- MAX aggregator
def brute_max(h_ids, z, br, dout=None, act="none", join_dst=True, concat_dst=True):
    """Per-key, per-feature maximum of the brute-force tuple outputs with explicit loops, the winner
    being the first tuple attaining it when a key's tuples are listed by (dst H row, E row, src H
    row); with ``dout`` (rows in key order) also the gradients (dW, db, dz) by explicit loops."""
    per_key = {}
    for (e, a, c) in brute_join(br.src, br.dst, h_ids, join_dst):
        x = list(z[a]) + (list(z[c]) if concat_dst else [])
        pre = [br.b[o] + sum(br.W[o][k] * x[k] for k in range(len(x))) for o in range(len(br.W))]
        y = [v if (act != "relu" or v > 0) else 0.0 for v in pre]
        per_key.setdefault(br.dst[e], []).append(((c, e, a), x, pre, y, a, c))
    keys = sorted(per_key)
    d_out, d_in, d = len(br.W), len(br.W[0]), z.shape[1]
    out = np.zeros((len(keys), d_out))
    dW, db, dz = np.zeros((d_out, d_in)), np.zeros(d_out), np.zeros_like(z)
    for i, k in enumerate(keys):
        tuples = sorted(per_key[k], key=lambda t: t[0])
        for o in range(d_out):
            best = None
            for t in tuples:
                if best is None or t[3][o] > best[3][o]:
                    best = t
            out[i, o] = best[3][o]
            if dout is None or (act == "relu" and not best[2][o] > 0):
                continue
            g = dout[i][o]
            _, x, _, _, a, c = best
            db[o] += g
            for kk in range(d_in):
                dW[o][kk] += g * x[kk]
                if kk < d:
                    dz[a][kk] += g * br.W[o][kk]
                elif concat_dst:
                    dz[c][kk - d] += g * br.W[o][kk]
    return keys, out, (dW, db, dz)


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("act", ["none", "relu"])
def test_max_matches_brute_force(seed, act):
    h_ids, z, br = tiny(seed + 100, n_e=50)
    keys, out, _ = O.rule_forward(h_ids, z, [br], act=act, agg="max")
    C = np.random.default_rng(seed).standard_normal(out.shape)
    bk, bo, (bW, bb, bz) = brute_max(h_ids, z, br, C, act)
    assert list(keys) == bk
    np.testing.assert_allclose(out, bo, rtol=1e-12, atol=1e-12)
    dW, db, dz, _ = O.rule_backward(h_ids, z, [br], keys, C, act=act, agg="max")
    np.testing.assert_allclose(dW[0], bW, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(db[0], bb, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(dz, bz, rtol=1e-12, atol=1e-12)


def test_max_brute_force_with_ties():
    """Quantised inputs make many tuples tie; the brute-force walk (first in the tie order wins)
    and the oracle must still agree exactly, also without a dst join (readout form)."""
    h_ids, z, br = tiny(110, n_e=80, n_h=14)
    rng = np.random.default_rng(3)
    z[:] = rng.integers(-2, 3, size=z.shape)
    br.W = rng.integers(-1, 2, size=br.W.shape).astype(float)
    br.b = np.zeros(br.W.shape[0])
    for join_dst in (True, False):
        b2 = Br(br.src, br.dst, br.W if join_dst else br.W[:, :z.shape[1]], br.b)
        keys, out, _ = O.rule_forward(h_ids, z, [b2], act="relu", join_dst=join_dst, concat_dst=join_dst,
                                      agg="max")
        C = rng.integers(-3, 4, size=out.shape).astype(float)
        bk, bo, (bW, bb, bz) = brute_max(h_ids, z, b2, C, "relu", join_dst, join_dst)
        assert list(keys) == bk
        assert np.array_equal(out, bo)
        dW, db, dz, _ = O.rule_backward(h_ids, z, [b2], keys, C, act="relu", join_dst=join_dst,
                                        concat_dst=join_dst, agg="max")
        assert np.array_equal(dW[0], bW) and np.array_equal(db[0], bb) and np.array_equal(dz, bz)


def test_max_tie_goes_to_the_first_tuple_by_hand():
    """Hand-derived: d = 1, W = [[1, 0]], b = 0, so y = z[src row].
    H rows: 0 key 9 (z 1), 1 key 9 (z 1), 2 key 1 (z 0), 3 key 2 (z 5), 4 key 1 (z 5).
    E: e0 = (1, 9), e1 = (2, 9). Key 9's tuples (dst row, E row, src row): (0,0,2) y 0, (0,0,4) y 5,
    (0,1,3) y 5, (1,0,2) y 0, (1,0,4) y 5, (1,1,3) y 5. Max 5; the first in that order is
    (dst 0, e0, src 4), so with dOut = 2: dz[4] = 2 * W[0][0] = 2, dz[0] = 2 * W[0][1] = 0, every
    other row 0; dW = 2 * x = [[10, 2]], db = [2]. An order that put the src row before the E row
    would pick (0, 1, 3) and send the gradient to row 3; the last occurrence would pick (1, 1, 3)."""
    h_ids = np.array([9, 9, 1, 2, 1])
    z = np.array([[1.0], [1.0], [0.0], [5.0], [5.0]])
    br = Br(np.array([1, 2]), np.array([9, 9]), np.array([[1.0, 0.0]]), np.array([0.0]))
    keys, out, _ = O.rule_forward(h_ids, z, [br], agg="max")
    assert keys.tolist() == [9] and out.tolist() == [[5.0]]
    dW, db, dz, _ = O.rule_backward(h_ids, z, [br], keys, np.array([[2.0]]), agg="max")
    assert dW[0].tolist() == [[10.0, 2.0]] and db[0].tolist() == [2.0]
    assert dz[:, 0].tolist() == [0.0, 0.0, 0.0, 0.0, 2.0]


def test_max_of_single_tuple_rows_is_sum():
    """Keys that receive exactly one tuple: MAX = SUM, forward and backward."""
    rng = np.random.default_rng(12)
    h_ids = np.arange(30)
    z = rng.standard_normal((30, 3))
    br = Br(rng.integers(0, 30, size=25), rng.permutation(30)[:25], rng.standard_normal((4, 6)),
            rng.standard_normal(4))
    k1, o1, _ = O.rule_forward(h_ids, z, [br], act="relu", agg="max")
    k2, o2, _ = O.rule_forward(h_ids, z, [br], act="relu")
    assert np.array_equal(k1, k2)
    np.testing.assert_allclose(o1, o2, rtol=1e-12, atol=1e-12)
    C = rng.standard_normal(o1.shape)
    g1 = O.rule_backward(h_ids, z, [br], k1, C, act="relu", agg="max")
    g2 = O.rule_backward(h_ids, z, [br], k2, C, act="relu")
    for a, b in ((g1[0][0], g2[0][0]), (g1[1][0], g2[1][0]), (g1[2], g2[2])):
        np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12)


def test_max_bounds_every_member_and_is_attained():
    h_ids, z, br = tiny(120, n_e=60)
    keys, out, _ = O.rule_forward(h_ids, z, [br], agg="max")
    e, hs, hd = O.join(br.src, br.dst, h_ids)
    Y = O.concat_rows(z, None, e, hs, hd) @ br.W.T + br.b
    gk = np.asarray(br.dst)[e]
    for i, k in enumerate(keys.tolist()):
        Yk = Y[gk == k]
        assert np.all(Yk <= out[i] + 0.0)
        assert np.all(np.any(Yk == out[i], axis=0))


@pytest.mark.parametrize("act", ["none", "relu"])
def test_max_backward_finite_differences(act):
    """MAX is piecewise linear: away from ties (continuous random inputs) central differences with a
    small step reproduce the backward exactly up to rounding."""
    h_ids, z, br = tiny(130, n_e=30, n_h=10, d=3, d_out=4)
    keys, out, _ = O.rule_forward(h_ids, z, [br], act=act, agg="max")
    C = np.random.default_rng(9).standard_normal(out.shape)
    dW, db, dz, _ = O.rule_backward(h_ids, z, [br], keys, C, act=act, agg="max")
    h = 1e-6

    def loss():
        return float(np.sum(O.rule_forward(h_ids, z, [br], act=act, agg="max")[1] * C))

    rng = np.random.default_rng(13)
    for arr, grad in ((br.W, dW[0]), (br.b, db[0]), (z, dz)):
        for _ in range(5):
            i = tuple(rng.integers(0, s) for s in arr.shape)
            old = arr[i]
            arr[i] = old + h
            lp = loss()
            arr[i] = old - h
            lm = loss()
            arr[i] = old
            assert (lp - lm) / (2 * h) == pytest.approx(grad[i], rel=1e-6, abs=1e-7)


# ----------------------------------------------------------------------------- attention over a join
def _attn_case(seed, n_h=12, n_e=50, d=8, key_range=10, dup=True):
    rng = np.random.default_rng(seed)
    h_ids = rng.integers(0, key_range, size=n_h) if dup else rng.permutation(key_range)[:n_h]
    q, k, v = (rng.standard_normal((n_h, d)) for _ in range(3))
    src = rng.integers(0, key_range + 2, size=n_e)
    dst = rng.integers(0, key_range + 2, size=n_e)
    return h_ids, q, k, v, src, dst


def brute_attention(h_ids, q, k, v, src, dst, n_heads, scale, mode):
    """Explicit loops over E x H x H: per output key, the list of (q row, k row, v row) of its
    tuples, then the product head or the per-head softmax written out term by term."""
    groups = {}
    for (e, a, c) in brute_join(src, dst, h_ids):
        groups.setdefault(dst[e], []).append((c, a))
    keys = sorted(groups)
    d, d_v = q.shape[1], v.shape[1]
    out = np.zeros((len(keys), d_v))
    for i, key in enumerate(keys):
        tuples = groups[key]
        if mode == "product":
            for (c, a) in tuples:
                for f in range(d_v):
                    out[i][f] += q[c][f] * k[a][f] * v[a][f]
            continue
        hq, hv = d // n_heads, d_v // n_heads
        for h in range(n_heads):
            sc = []
            for (c, a) in tuples:
                sc.append(scale * sum(q[c][h * hq + j] * k[a][h * hq + j] for j in range(hq)))
            mx = max(sc)
            w = [np.exp(x - mx) for x in sc]
            tot = sum(w)
            for (c, a), wt in zip(tuples, w):
                for j in range(hv):
                    out[i][h * hv + j] += wt / tot * v[a][h * hv + j]
    return keys, out


@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("mode,heads", [("product", 1), ("softmax", 1), ("softmax", 2), ("softmax", 4)])
def test_attention_matches_brute_force(seed, mode, heads):
    h_ids, q, k, v, src, dst = _attn_case(seed + 200)
    keys, out, _ = O.attention_forward(h_ids, q, k, v, src, dst, heads, 0.7, mode)
    bk, bo = brute_attention(h_ids, q, k, v, src, dst, heads, 0.7, mode)
    assert list(keys) == bk
    np.testing.assert_allclose(out, bo, rtol=1e-12, atol=1e-12)


def test_attention_uniform_weights_is_the_mean_aggregator():
    """k = 0 makes every score 0, so the softmax weights are uniform: the output is the MEAN of the
    group's v rows, i.e. the identity rule with alpha = MEAN over z = v (no z_dst)."""
    h_ids, q, k, v, src, dst = _attn_case(210)
    keys, out, _ = O.attention_forward(h_ids, q, np.zeros_like(k), v, src, dst, 2, 1.0, "softmax")
    br = Br(src, dst, None, None)
    k2, mean, _ = O.rule_forward(h_ids, v, [br], concat_dst=False, agg="mean")
    assert np.array_equal(keys, k2)
    np.testing.assert_allclose(out, mean, rtol=1e-12, atol=1e-12)


def test_attention_is_invariant_to_a_shift_of_the_keys():
    """With unique H keys every tuple of output key p uses the same q row, so adding one vector c to
    every k row shifts all of p's scores by the same scale * q_p . c: the softmax is unchanged."""
    h_ids, q, k, v, src, dst = _attn_case(211, dup=False)
    c = np.random.default_rng(1).standard_normal(k.shape[1])
    _, o1, _ = O.attention_forward(h_ids, q, k, v, src, dst, 2, 0.5)
    _, o2, _ = O.attention_forward(h_ids, q, k + c, v, src, dst, 2, 0.5)
    np.testing.assert_allclose(o1, o2, rtol=1e-10, atol=1e-12)


def test_attention_single_tuple_keys_return_v():
    rng = np.random.default_rng(4)
    h_ids = np.arange(30)
    q, k, v = (rng.standard_normal((30, 8)) for _ in range(3))
    src, dst = rng.integers(0, 30, size=20), rng.permutation(30)[:20]
    keys, out, lse = O.attention_forward(h_ids, q, k, v, src, dst, 4, 0.3)
    order = np.argsort(dst)
    np.testing.assert_allclose(out, v[src[order]], rtol=1e-12, atol=1e-12)
    s = 0.3 * (q[dst[order]] * k[src[order]]).reshape(20, 4, 2).sum(axis=2)
    np.testing.assert_allclose(lse, s, rtol=1e-12, atol=1e-12)  # log of a single exp


@pytest.mark.parametrize("mode,heads", [("product", 1), ("softmax", 2)])
def test_attention_backward_finite_differences(mode, heads):
    h_ids, q, k, v, src, dst = _attn_case(220, n_e=30, d=4)
    keys, out, _ = O.attention_forward(h_ids, q, k, v, src, dst, heads, 0.8, mode)
    C = np.random.default_rng(5).standard_normal(out.shape)
    dq, dk, dv = O.attention_backward(h_ids, q, k, v, src, dst, C, heads, 0.8, mode)
    h = 1e-6

    def loss():
        return float(np.sum(O.attention_forward(h_ids, q, k, v, src, dst, heads, 0.8, mode)[1] * C))

    rng = np.random.default_rng(6)
    for arr, grad in ((q, dq), (k, dk), (v, dv)):
        for _ in range(6):
            i = tuple(rng.integers(0, s) for s in arr.shape)
            old = arr[i]
            arr[i] = old + h
            lp = loss()
            arr[i] = old - h
            lm = loss()
            arr[i] = old
            assert (lp - lm) / (2 * h) == pytest.approx(grad[i], rel=1e-6, abs=1e-7)


# ----------------------------------------------------------------------------- triangle (cyclic) join
def _tri_case(seed, n_keys=9, n_e=40, n_h=11, d=3):
    rng = np.random.default_rng(seed)
    h_ids = rng.integers(0, n_keys, size=n_h)  # duplicate keys and keys without a row
    src = rng.integers(0, n_keys + 1, size=n_e)
    dst = rng.integers(0, n_keys + 1, size=n_e)
    a, b, c = (rng.standard_normal((n_h, d)) for _ in range(3))
    return h_ids, a, b, c, src, dst


@pytest.mark.parametrize("seed", range(4))
def test_triangle_matches_brute_force_over_edge_triples(seed):
    """Explicit loops over all E x E x E triples and the H rows of their three keys."""
    h_ids, a, b, c, src, dst = _tri_case(300 + seed)
    acc = {}
    E = list(zip(src.tolist(), dst.tolist()))
    for (n, v) in E:
        for (v2, w) in E:
            if v2 != v:
                continue
            for (w2, n2) in E:
                if w2 != w or n2 != n:
                    continue
                for ra in range(len(h_ids)):
                    if h_ids[ra] != n:
                        continue
                    for rb in range(len(h_ids)):
                        if h_ids[rb] != v:
                            continue
                        for rc in range(len(h_ids)):
                            if h_ids[rc] != w:
                                continue
                            acc[n] = acc.get(n, 0) + a[ra] * b[rb] * c[rc]
    keys, out = O.triangle_forward(h_ids, a, b, c, src, dst)
    assert list(keys) == sorted(acc)
    np.testing.assert_allclose(out, np.array([acc[k] for k in sorted(acc)]).reshape(out.shape), rtol=1e-12,
                               atol=1e-12)


def test_triangle_closed_form_diag_of_matrix_products():
    """With unique H keys 0..K-1, feature f of Out[n] is a_n * (M D_b M D_c M)[n][n], where M is
    the edge multiplicity matrix and D_x = diag(x[:, f]): a closed form independent of the walk."""
    rng = np.random.default_rng(11)
    K = 12
    h_ids = np.arange(K)
    src, dst = rng.integers(0, K, size=70), rng.integers(0, K, size=70)
    a, b, c = (rng.standard_normal((K, 2)) for _ in range(3))
    M = np.zeros((K, K))
    np.add.at(M, (src, dst), 1.0)
    keys, out = O.triangle_forward(h_ids, a, b, c, src, dst)
    for f in range(2):
        diag = np.diag(M @ np.diag(b[:, f]) @ M @ np.diag(c[:, f]) @ M) * a[:, f]
        nz = np.nonzero(np.diag(M @ M @ M))[0]
        np.testing.assert_allclose(out[:, f], diag[keys], rtol=1e-12, atol=1e-12)
        assert set(keys.tolist()) == set(nz.tolist())


def test_triangle_counts_with_unit_embeddings():
    """a = b = c = 1, d = 1: Out[n] counts the closed directed 3-walks from n, edge multiplicities
    multiplying. Hand graph: the 3-cycle 0->1->2->0 with the edge 1->2 doubled gives 2 matches at
    each of 0, 1 and 2 (either copy of 1->2), and the self-loop 3->3 gives 1 match at 3."""
    h_ids = np.arange(4)
    src = np.array([0, 1, 1, 2, 3])
    dst = np.array([1, 2, 2, 0, 3])
    ones = np.ones((4, 1))
    keys, out = O.triangle_forward(h_ids, ones, ones, ones, src, dst)
    assert keys.tolist() == [0, 1, 2, 3]
    assert out[:, 0].tolist() == [2.0, 2.0, 2.0, 1.0]


def test_triangle_backward_finite_differences():
    h_ids, a, b, c, src, dst = _tri_case(320, n_e=50)
    keys, out = O.triangle_forward(h_ids, a, b, c, src, dst)
    C = np.random.default_rng(2).standard_normal(out.shape)
    da, db, dc = O.triangle_backward(h_ids, a, b, c, src, dst, C)
    h = 1e-6

    def loss():
        return float(np.sum(O.triangle_forward(h_ids, a, b, c, src, dst)[1] * C))

    rng = np.random.default_rng(3)
    for arr, grad in ((a, da), (b, db), (c, dc)):
        for _ in range(6):
            i = tuple(rng.integers(0, s) for s in arr.shape)
            old = arr[i]
            arr[i] = old + h
            lp = loss()
            arr[i] = old - h
            lm = loss()
            arr[i] = old
            assert (lp - lm) / (2 * h) == pytest.approx(grad[i], rel=1e-6, abs=1e-7)
