"""FP64 CPU oracle for RelaNN rule evaluation -- TEST INFRASTRUCTURE ONLY.

This module is the plain, slow, obviously-correct definition of what the GPU path computes. Only the
test suite, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of ``bench.py`` may
import it; the library never does. It shares no code with the CUDA path.

Every floating-point step runs in float64. Inputs that the device holds in bf16 are passed in after
rounding to bf16 (an exact upcast), so both sides see the same values.

Definitions followed (paper sections):
  * embedded relation (r, eta): content tuples plus one embedding per tuple          -- Sec. 2.1
  * join: natural join on shared attributes; embedding = concatenation eta1 (+) eta2   -- Sec. 2.2
  * projected union with aggregator alpha: group by the projected key, alpha over the
    multiset B_t of contributing tuples (alpha = SUM, MEAN = SUM / |B_t|, or MAX per
    feature; the union compiles to a scatter reduction chosen by alpha)              -- Sec. 2.2, 4.2
  * transformation T_tau: tau applied to each tuple embedding independently            -- Sec. 2.2
  * selection: a conjunctive filter expression of atomic predicates e1 theta e2 over the
    body's content variables (here a tuple's src and dst keys) and constants; a tuple
    that fails it does not take part in the join                                       -- Sec. 3.1, 4.2
  * join rule R(x; alpha(tau)) :- R1,...,Rk  ==  U_{alpha,x}(T_tau(R1 |><| ... |><| Rk)) -- Sec. 3.1
  * union rule / "|..." replicator: branch results added by the head's sum             -- Sec. 3.1, 3.7
  * fit: parameters (weights and per-tuple embeddings) minimise a loss relation        -- Sec. 2.3, 3.2, 3.6
  * attention over a join: Score(p, t; q*k) :- E(t, p), Q(p; q), K(t; k) and
    Attention(p; sum(a*v)) :- Score(p, t; a), V(t; v) (element-wise product head), and the
    HGT head: per head, softmax over t of the scaled dot product q . k, then the weighted
    sum of v                                                                          -- Sec. 1, Sec. 5 (HGT)
  * cyclic self-join (DHN triangle homomorphisms): Out(n; sum(a_n * b_v * c_w)) :-
    E(n, v), E(v, w), E(w, n), H(n; a), H(v; b), H(w; c), element-wise products      -- Sec. 5 (DHN)

Readings where the paper is silent (each is listed with its reason in the design notes):
  * bag semantics: every E row is a distinct tuple, duplicate H keys each match;
  * a tuple whose key is absent from H is dropped by the join;
  * output keys are exactly the keys with >= 1 contributing tuple, sorted ascending;
  * Concat order is (z_src, z_dst[, r_edge]); Linear is y = x W^T + b with W [d_out, d_in];
  * ReLU (when present) is applied per tuple, inside the SUM.
  * MAX: the gradient of a row's maximum goes to one tuple, the first that attains it in the
    order (dst H row, E row, src H row) within the row; ReLU' is taken at that tuple.

Parity status: every function here is pinned by ``tests/test_oracle.py`` (nested-loop brute force,
closed forms, invariants, finite differences, a hand-derived golden fixture).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "key_index", "join", "join_pairs", "join_cardinality", "concat_rows", "group_sum", "group_max",
    "max_tie_order", "selected_rows",
    "selected_join",
    "rule_forward", "rule_backward", "mse", "mse_grad", "stacked_forward", "stacked_backward",
    "attention_forward", "attention_backward", "triangle_forward", "triangle_backward",
]

CHUNK = 1 << 20  # join triples processed per NumPy block in the Linear/SUM steps


def key_index(h_ids) -> dict:
    """Key -> list of H row numbers, in row order (a bag: every duplicate row is kept). Sec. 2.2."""
    idx: dict = {}
    for row, k in enumerate(np.asarray(h_ids).tolist()):
        idx.setdefault(k, []).append(row)
    return idx


def join_pairs(probe_keys, build_keys):
    """One-sided equi-join P(k) |><| B(k) under bag semantics (Sec. 2.2 Join).

    Returns int64 arrays (probe_row, build_row), ordered by probe row then build row."""
    idx = key_index(build_keys)
    pr, br = [], []
    for i, k in enumerate(np.asarray(probe_keys).tolist()):
        rows = idx.get(k)
        if rows:
            for b in rows:
                pr.append(i)
                br.append(b)
    return np.asarray(pr, np.int64), np.asarray(br, np.int64)


def join(src, dst, h_ids, join_dst: bool = True):
    """E(src, dst) |><| H(src) [|><| H(dst)] under bag semantics (Sec. 2.2 Join, Sec. 3.1 rule body).

    Returns int64 arrays (e, hs, hd): one entry per join output tuple, ordered by E row, then the
    src-side H row, then the dst-side H row. With ``join_dst`` false the dst key is carried as
    content only and hd is -1."""
    idx = key_index(h_ids)
    e_l, hs_l, hd_l = [], [], []
    none = [-1]
    for e, (s, d) in enumerate(zip(np.asarray(src).tolist(), np.asarray(dst).tolist())):
        rs = idx.get(s)
        if not rs:
            continue
        rd = idx.get(d) if join_dst else none
        if not rd:
            continue
        for a in rs:
            for b in rd:
                e_l.append(e)
                hs_l.append(a)
                hd_l.append(b)
    return (np.asarray(e_l, np.int64), np.asarray(hs_l, np.int64), np.asarray(hd_l, np.int64))


def join_cardinality(src, dst, h_ids, join_dst: bool = True) -> int:
    """|E |><| H |><| H| = sum over E rows of cnt_H(src) * cnt_H(dst) (bag semantics)."""
    cnt: dict = {}
    for k in np.asarray(h_ids).tolist():
        cnt[k] = cnt.get(k, 0) + 1
    total = 0
    for s, d in zip(np.asarray(src).tolist(), np.asarray(dst).tolist()):
        total += cnt.get(s, 0) * (cnt.get(d, 0) if join_dst else 1)
    return total


def concat_rows(z, r, e, hs, hd, concat_dst: bool = True):
    """X_t = z[hs_t] (+) z[hd_t] (+) r[e_t] in float64 (Sec. 2.2 Join embedding semantics)."""
    z = np.asarray(z, np.float64)
    parts = [z[hs]]
    if concat_dst:
        parts.append(z[hd])
    if r is not None:
        parts.append(np.asarray(r, np.float64)[e])
    return np.concatenate(parts, axis=1)


def group_sum(keys, values):
    """Projected union with alpha = SUM (Sec. 2.2): sorted distinct keys and per-key sums."""
    uk, inv = np.unique(np.asarray(keys), return_inverse=True)
    out = np.zeros((uk.size, values.shape[1]), np.float64)
    np.add.at(out, inv.reshape(-1), values)
    return uk, out


def max_tie_order(keys, e, hs, hd):
    """Permutation listing the join triples by output key, and within a key by dst H row, then E
    row, then src H row: the order in which MAX keeps the first tuple attaining a maximum."""
    return np.lexsort((np.asarray(hs), np.asarray(e), np.asarray(hd), np.asarray(keys)))


def group_max(keys, values, order):
    """Projected union with alpha = MAX (Sec. 2.2), per column. ``order`` lists the rows of
    ``values`` grouped by key (``max_tie_order``). Returns the sorted distinct keys, the per-key
    column maxima, and for each (key, column) the row that attains the maximum first in ``order``."""
    order = np.asarray(order, np.int64)
    k_sorted = np.asarray(keys)[order]
    uk, start = np.unique(k_sorted, return_index=True)
    bounds = list(start) + [order.size]
    n_col = values.shape[1]
    out = np.zeros((uk.size, n_col), np.float64)
    win = np.zeros((uk.size, n_col), np.int64)
    cols = np.arange(n_col)
    for g in range(uk.size):
        rows = order[bounds[g]:bounds[g + 1]]
        block = values[rows]
        first = np.argmax(block, axis=0)  # the first occurrence of each column's maximum
        out[g] = block[first, cols]
        win[g] = rows[first]
    return uk, out, win


def _tau(X, W, b, act):
    """T_tau with tau = [ReLU o] Linear (Sec. 2.2 Transformation): y = x W^T + b per tuple."""
    if W is None:
        Y = X.copy()
    else:
        Y = X @ np.asarray(W, np.float64).T
        if b is not None:
            Y = Y + np.asarray(b, np.float64)
    if act == "relu":
        Y = np.maximum(Y, 0.0)
    return Y


_CMP = {"==": np.equal, "!=": np.not_equal, "<": np.less, "<=": np.less_equal, ">": np.greater,
        ">=": np.greater_equal}


def selected_rows(br):
    """Boolean mask of the E rows that satisfy the branch's filter expression (all predicates;
    ``br.filters`` is absent or a list of (lhs, op, rhs), lhs / rhs = "src", "dst" or an int)."""
    src = np.asarray(br.src)
    keep = np.ones(src.size, bool)
    for lhs, op, rhs in getattr(br, "filters", None) or []:
        def term(x):
            if isinstance(x, str):
                return np.asarray({"src": br.src, "dst": br.dst}[x]).astype(np.int64)
            return np.int64(x)
        keep &= _CMP[op](term(lhs), term(rhs))
    return keep


def selected_join(br, h_ids, join_dst):
    """The join triples (e, hs, hd) of the branch's E rows that pass its selection."""
    e, hs, hd = join(br.src, br.dst, h_ids, join_dst)
    keep = selected_rows(br)[e]
    return e[keep], hs[keep], hd[keep]


def rule_forward(h_ids, z, branches, act: str = "none", join_dst: bool = True,
                 concat_dst: bool = True, agg: str = "sum"):
    """Evaluate H'(dst; alpha(tau(Concat(...)))) :- E_i(src, dst[; r]), H(src; z_src), H(dst; z_dst)
    for every branch i and add the branch results (Sec. 3.1 join rule; union rule and the "|..."
    replicator of Sec. 3.7 for several branches). alpha = SUM, or MEAN: each branch's per-key sum
    divided by that branch's number of contributing tuples of the key (Sec. 2.2).

    ``branches``: sequence of objects with fields src, dst, r (or None), W (or None = identity), b.
    Returns (out_keys sorted ascending, out_z float64 [n_out, d_out], join sizes per branch)."""
    assert agg in ("sum", "mean", "max")
    if agg == "max":
        keys, out, _, sizes = _max_forward(h_ids, z, branches, act, join_dst, concat_dst)
        return keys, out, sizes
    acc: dict = {}
    sizes = []
    for br in branches:
        e, hs, hd = selected_join(br, h_ids, join_dst)
        sizes.append(int(e.size))
        dst = np.asarray(br.dst)
        bacc: dict = {}
        bcnt: dict = {}
        for lo in range(0, e.size, CHUNK):
            sl = slice(lo, lo + CHUNK)
            X = concat_rows(z, br.r, e[sl], hs[sl], hd[sl], concat_dst)
            Y = _tau(X, br.W, br.b, act)
            uk, part = group_sum(dst[e[sl]], Y)
            ck, cn = np.unique(dst[e[sl]], return_counts=True)
            for k, c in zip(ck.tolist(), cn.tolist()):
                bcnt[k] = bcnt.get(k, 0) + c
            for k, row in zip(uk.tolist(), part):
                bacc[k] = bacc[k] + row if k in bacc else row
        for k, row in bacc.items():
            if agg == "mean":
                row = row / bcnt[k]
            acc[k] = acc[k] + row if k in acc else row
    keys = sorted(acc)
    d_out = _out_dim(z, branches, concat_dst)
    out = np.stack([acc[k] for k in keys]) if keys else np.zeros((0, d_out))
    key_dtype = np.asarray(h_ids).dtype if join_dst else np.asarray(branches[0].dst).dtype
    return np.asarray(keys, key_dtype), out, sizes


def _max_forward(h_ids, z, branches, act, join_dst, concat_dst):
    """alpha = MAX for a single-branch rule: per output key and feature, the maximum of tau over the
    key's join tuples. Also returns the winners (row of the join triples per key and feature) and the
    triples, for the backward."""
    assert len(branches) == 1, "MAX: single-branch rules"
    br = branches[0]
    e, hs, hd = selected_join(br, h_ids, join_dst)
    dst = np.asarray(br.dst)
    X = concat_rows(z, br.r, e, hs, hd, concat_dst)
    Y = _tau(X, br.W, br.b, act)
    gk = dst[e]
    uk, out, win = group_max(gk, Y, max_tie_order(gk, e, hs, hd))
    if uk.size == 0:
        out = np.zeros((0, _out_dim(z, branches, concat_dst)))
    key_dtype = np.asarray(h_ids).dtype if join_dst else dst.dtype
    return np.asarray(uk, key_dtype), out, (win, e, hs, hd, X), [int(e.size)]


def _out_dim(z, branches, concat_dst):
    br = branches[0]
    if br.W is not None:
        return int(np.asarray(br.W).shape[0])
    d = np.asarray(z).shape[1] * (2 if concat_dst else 1)
    return d + (0 if br.r is None else np.asarray(br.r).shape[1])


def rule_backward(h_ids, z, branches, dout_keys, dout, act: str = "none", join_dst: bool = True,
                  concat_dst: bool = True, agg: str = "sum"):
    """Chain rule through the rule of ``rule_forward`` in float64 (the fit of Sec. 2.3 optimises the
    weights and the per-tuple embeddings, Sec. 3.6).

    SUM backward broadcasts dOut[dst] to every contributing tuple (MEAN: dOut[dst] divided by the
    branch's number of contributing tuples of dst); ReLU masks by the recomputed
    pre-activation; Linear gives dW = dY^T X, db = sum dY, dX = dY W; Concat backward splits dX and
    adds each slice to the embedding row it was gathered from.

    Returns (dW list, db list, dz [n_h, d], dr list (None where a branch has no r))."""
    z64 = np.asarray(z, np.float64)
    d = z64.shape[1]
    dz = np.zeros_like(z64)
    pos = {k: i for i, k in enumerate(np.asarray(dout_keys).tolist())}
    dout = np.asarray(dout, np.float64)
    if agg == "max":
        return _max_backward(h_ids, z64, branches[0], pos, dout, act, join_dst, concat_dst)
    dWs, dbs, drs = [], [], []
    for br in branches:
        e, hs, hd = selected_join(br, h_ids, join_dst)
        dst = np.asarray(br.dst)
        W = None if br.W is None else np.asarray(br.W, np.float64)
        dW = None if W is None else np.zeros_like(W)
        db = None if W is None else np.zeros(W.shape[0])
        dr = None if br.r is None else np.zeros(np.asarray(br.r).shape, np.float64)
        if agg == "mean":
            ck, cn = np.unique(dst[e], return_counts=True)
            cnt = dict(zip(ck.tolist(), cn.tolist()))
        for lo in range(0, e.size, CHUNK):
            sl = slice(lo, lo + CHUNK)
            X = concat_rows(z, br.r, e[sl], hs[sl], hd[sl], concat_dst)
            rows = np.asarray([pos[k] for k in dst[e[sl]].tolist()], np.int64)
            G = dout[rows]
            if agg == "mean":
                G = G / np.asarray([cnt[k] for k in dst[e[sl]].tolist()], np.float64)[:, None]
            if act == "relu":
                pre = _tau(X, W, br.b, "none")
                G = G * (pre > 0.0)
            if W is not None:
                dW += G.T @ X
                db += G.sum(axis=0)
                dX = G @ W
            else:
                dX = G
            np.add.at(dz, hs[sl], dX[:, :d])
            off = d
            if concat_dst:
                np.add.at(dz, hd[sl], dX[:, d:2 * d])
                off = 2 * d
            if dr is not None:
                np.add.at(dr, e[sl], dX[:, off:])
        dWs.append(dW)
        dbs.append(db)
        drs.append(dr)
    return dWs, dbs, dz, drs


def _max_backward(h_ids, z64, br, pos, dout, act, join_dst, concat_dst):
    """MAX backward: dOut[k][o] goes to the winner of (k, o) alone (ReLU' taken there)."""
    uk, _, (win, e, hs, hd, X), _ = _max_forward(h_ids, z64, [br], act, join_dst, concat_dst)
    W = None if br.W is None else np.asarray(br.W, np.float64)
    G = np.zeros((e.size, W.shape[0] if W is not None else X.shape[1]))
    for g, k in enumerate(uk.tolist()):
        G[win[g], np.arange(win.shape[1])] = dout[pos[k]]
    if act == "relu":
        G = G * (_tau(X, W, br.b, "none") > 0.0)
    d = z64.shape[1]
    dz = np.zeros_like(z64)
    dW = db = None
    if W is not None:
        dW = G.T @ X
        db = G.sum(axis=0)
        dX = G @ W
    else:
        dX = G
    np.add.at(dz, hs, dX[:, :d])
    off = d
    if concat_dst:
        np.add.at(dz, hd, dX[:, d:2 * d])
        off = 2 * d
    dr = None
    if br.r is not None:
        dr = np.zeros(np.asarray(br.r).shape, np.float64)
        np.add.at(dr, e, dX[:, off:])
    return [dW], [db], dz, [dr]


def mse(pred_keys, pred, target_keys, target):
    """Loss relation L(; mean((zp - zt)^2)) :- Pred(g; zp), Target(g; zt): a join on g, then the
    mean over every embedding cell of the joined pairs (Sec. 3.2 loss relation of arity 0)."""
    pos = {k: i for i, k in enumerate(np.asarray(target_keys).tolist())}
    pairs = [(i, pos[k]) for i, k in enumerate(np.asarray(pred_keys).tolist()) if k in pos]
    if not pairs:
        return 0.0
    p = np.asarray(pred, np.float64)[[a for a, _ in pairs]]
    t = np.asarray(target, np.float64)[[b for _, b in pairs]]
    return float(np.mean((p - t) ** 2))


def mse_grad(pred_keys, pred, target_keys, target):
    """d mse / d pred (rows of pred that join no target get zero gradient)."""
    pos = {k: i for i, k in enumerate(np.asarray(target_keys).tolist())}
    pred = np.asarray(pred, np.float64)
    g = np.zeros_like(pred)
    rows = [(i, pos[k]) for i, k in enumerate(np.asarray(pred_keys).tolist()) if k in pos]
    n = len(rows) * pred.shape[1]
    for i, j in rows:
        g[i] = 2.0 * (pred[i] - np.asarray(target[j], np.float64)) / n
    return g


class _Br:
    """Plain branch record (src, dst, r, W, b) for the stacked program."""

    def __init__(self, src, dst, W, b, r=None):
        self.src, self.dst, self.W, self.b, self.r = src, dst, W, b, r


def stacked_forward(h_ids, z, src, dst, W1, b1, W2, b2, g_keys, g_groups, t_groups, targets):
    """Two stacked rules and a SUM readout with an MSE loss:

        H1(d; SUM ReLU(Linear1(Concat(z_s, z_d)))) :- E(s, d), H(s; z_s), H(d; z_d)
        H2(d; SUM Linear2(Concat(z_s, z_d)))       :- E(s, d), H1(s; z_s), H1(d; z_d)
        Out(g; SUM z)                              :- H2(k; z), G(k, g)
        L(; mean((z_o - z_t)^2))                   :- Out(g; z_o), T(g; z_t)

    Returns a dict with every intermediate relation and the loss."""
    k1, h1, _ = rule_forward(h_ids, z, [_Br(src, dst, W1, b1)], act="relu")
    k2, h2, _ = rule_forward(k1, h1, [_Br(src, dst, W2, b2)], act="none")
    ko, ho, _ = rule_forward(k2, h2, [_Br(g_keys, g_groups, None, None)], join_dst=False,
                             concat_dst=False)
    loss = mse(ko, ho, t_groups, targets)
    return dict(k1=k1, h1=h1, k2=k2, h2=h2, ko=ko, ho=ho, loss=loss)


def stacked_backward(h_ids, z, src, dst, W1, b1, W2, b2, g_keys, g_groups, t_groups, targets,
                     fwd=None):
    """Analytic float64 gradient of ``stacked_forward``'s loss w.r.t. W1, b1, W2, b2 and z."""
    f = fwd if fwd is not None else stacked_forward(h_ids, z, src, dst, W1, b1, W2, b2, g_keys,
                                                    g_groups, t_groups, targets)
    d_ho = mse_grad(f["ko"], f["ho"], t_groups, targets)
    _, _, d_h2, _ = rule_backward(f["k2"], f["h2"], [_Br(g_keys, g_groups, None, None)], f["ko"],
                                  d_ho, join_dst=False, concat_dst=False)
    (dW2,), (db2,), d_h1, _ = rule_backward(f["k1"], f["h1"], [_Br(src, dst, W2, b2)], f["k2"], d_h2)
    (dW1,), (db1,), dz, _ = rule_backward(h_ids, z, [_Br(src, dst, W1, b1)], f["k1"], d_h1,
                                          act="relu")
    return dict(dW1=dW1, db1=db1, dW2=dW2, db2=db2, dz=dz, d_h1=d_h1, d_h2=d_h2, d_ho=d_ho)


# ----------------------------------------------------------------------------- attention over a join
def _attn_parts(h_ids, src, dst):
    """Join triples of E(t = src, p = dst) with H on both sides; the output key of a tuple is p."""
    e, hs, hd = join(src, dst, h_ids)
    keys = np.asarray(dst)[e]
    uk, inv = np.unique(keys, return_inverse=True)
    return e, hs, hd, uk, inv.reshape(-1)


def _scores(q, k, hs, hd, n_heads, scale):
    """s[t, h] = scale * sum over head h's features of q[hd_t] * k[hs_t]."""
    d = q.shape[1]
    prod = (q[hd] * k[hs]).reshape(hs.size, n_heads, d // n_heads)
    return scale * prod.sum(axis=2)


def attention_forward(h_ids, q, k, v, src, dst, n_heads=1, scale=1.0, mode="softmax"):
    """Attention of each output key p over its join tuples t (E rows with dst = p; q from the dst
    side's H row, k and v from the src side's H row), in float64.

    mode "product" (the Sec. 1 program): Out[p] = sum_t q_t * k_t * v_t element-wise (d_v = d).
    mode "softmax" (the HGT head of Sec. 5): per head h, a_t = exp(s_t) / sum_t' exp(s_t') with
    s_t = scale * q_t . k_t over the head's features, and Out[p][h] = sum_t a_t v_t[h].
    Returns (sorted output keys, Out [n_out, d_v], logsumexp [n_out, n_heads] or None)."""
    q = np.asarray(q, np.float64)
    k = np.asarray(k, np.float64)
    v = np.asarray(v, np.float64)
    e, hs, hd, uk, inv = _attn_parts(h_ids, src, dst)
    d_v = v.shape[1]
    out = np.zeros((uk.size, d_v))
    if mode == "product":
        np.add.at(out, inv, q[hd] * k[hs] * v[hs])
        return uk, out, None
    s = _scores(q, k, hs, hd, n_heads, scale)
    lse = np.full((uk.size, n_heads), -np.inf)
    for g in range(uk.size):
        rows = np.nonzero(inv == g)[0]
        sg = s[rows]
        m = sg.max(axis=0)
        w = np.exp(sg - m)
        lse[g] = m + np.log(w.sum(axis=0))
        a = w / w.sum(axis=0)
        vg = v[hs[rows]].reshape(rows.size, n_heads, d_v // n_heads)
        out[g] = (a[:, :, None] * vg).sum(axis=0).reshape(d_v)
    return uk, out, lse


def attention_backward(h_ids, q, k, v, src, dst, dout, n_heads=1, scale=1.0, mode="softmax"):
    """Gradients (dq, dk, dv) of sum(dout * Out) for ``attention_forward`` (rows of dout in its key
    order); each tuple's contribution is added to the H rows it was gathered from."""
    q = np.asarray(q, np.float64)
    k = np.asarray(k, np.float64)
    v = np.asarray(v, np.float64)
    dout = np.asarray(dout, np.float64)
    e, hs, hd, uk, inv = _attn_parts(h_ids, src, dst)
    dq, dk, dv = np.zeros_like(q), np.zeros_like(k), np.zeros_like(v)
    G = dout[inv]
    if mode == "product":
        np.add.at(dq, hd, G * k[hs] * v[hs])
        np.add.at(dk, hs, G * q[hd] * v[hs])
        np.add.at(dv, hs, G * q[hd] * k[hs])
        return dq, dk, dv
    _, out, lse = attention_forward(h_ids, q, k, v, src, dst, n_heads, scale, mode)
    d, d_v = q.shape[1], v.shape[1]
    s = _scores(q, k, hs, hd, n_heads, scale)
    a = np.exp(s - lse[inv])                                   # [T, heads]
    Gh = G.reshape(-1, n_heads, d_v // n_heads)
    vh = v[hs].reshape(-1, n_heads, d_v // n_heads)
    np.add.at(dv, hs, (a[:, :, None] * Gh).reshape(-1, d_v))
    da = (Gh * vh).sum(axis=2)                                 # dL/da_t per head
    D = (dout.reshape(-1, n_heads, d_v // n_heads) * out.reshape(-1, n_heads, d_v // n_heads)).sum(axis=2)
    ds = a * (da - D[inv]) * scale                             # dL/d(q . k) per head
    dsf = np.repeat(ds, d // n_heads, axis=1)
    np.add.at(dq, hd, dsf * k[hs])
    np.add.at(dk, hs, dsf * q[hd])
    return dq, dk, dv


# ----------------------------------------------------------------------------- triangle (cyclic) join
def triangle_matches(h_ids, src, dst):
    """All matches of E(n, v), E(v, w), E(w, n) joined with H on n, v and w (bag semantics: every E
    row is a tuple and every H row of a key matches). Returns int64 arrays (n_key, row_n, row_v,
    row_w), one entry per match, ordered by the three E rows (e1, e2, e3) then the H rows."""
    idx = key_index(h_ids)
    src = np.asarray(src).tolist()
    dst = np.asarray(dst).tolist()
    out_of: dict = {}
    for e, (a, b) in enumerate(zip(src, dst)):
        out_of.setdefault(a, []).append(e)
    keys, rn, rv, rw = [], [], [], []
    for e1, (n, v) in enumerate(zip(src, dst)):
        if n not in idx or v not in idx:
            continue
        for e2 in out_of.get(v, []):
            w = dst[e2]
            if w not in idx:
                continue
            for e3 in out_of.get(w, []):
                if dst[e3] != n:
                    continue
                for a in idx[n]:
                    for b in idx[v]:
                        for c in idx[w]:
                            keys.append(n)
                            rn.append(a)
                            rv.append(b)
                            rw.append(c)
    return (np.asarray(keys, np.int64), np.asarray(rn, np.int64), np.asarray(rv, np.int64),
            np.asarray(rw, np.int64))


def triangle_forward(h_ids, a, b, c, src, dst):
    """Out(n; sum(a_n * b_v * c_w)) over the triangle matches, grouped by the key of n (ascending;
    only keys with at least one match). Returns (keys, Out [n_out, d]) in float64."""
    a, b, c = (np.asarray(x, np.float64) for x in (a, b, c))
    keys, rn, rv, rw = triangle_matches(h_ids, src, dst)
    uk, inv = np.unique(keys, return_inverse=True)
    out = np.zeros((uk.size, a.shape[1]))
    np.add.at(out, inv.reshape(-1), a[rn] * b[rv] * c[rw])
    return uk.astype(np.asarray(h_ids).dtype), out


def triangle_backward(h_ids, a, b, c, src, dst, dout):
    """Gradients (da, db, dc) of sum(dout * Out) for ``triangle_forward`` (dout rows in its key order)."""
    a, b, c = (np.asarray(x, np.float64) for x in (a, b, c))
    keys, rn, rv, rw = triangle_matches(h_ids, src, dst)
    uk, inv = np.unique(keys, return_inverse=True)
    G = np.asarray(dout, np.float64)[inv.reshape(-1)]
    da, db, dc = np.zeros_like(a), np.zeros_like(b), np.zeros_like(c)
    np.add.at(da, rn, G * b[rv] * c[rw])
    np.add.at(db, rv, G * a[rn] * c[rw])
    np.add.at(dc, rw, G * a[rn] * b[rv])
    return da, db, dc
