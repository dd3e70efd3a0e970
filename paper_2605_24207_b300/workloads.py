"""Seeded synthetic relations shaped like the rule workloads (inputs only, no rule arithmetic).

This module is shared by the tests, the benchmark and the CPU checker: it draws keys, tuples and
embeddings and nothing else. Every array is NumPy on the host; callers move them to the device.

Readings used for the draws (the paper gives shapes, not distributions):
  * keys are K distinct integers; by default a seeded permutation of 0..K-1 stored in shuffled H
    row order (so key -> row is not the identity); ``sparse_keys`` draws K distinct values from a
    wide range instead (int64: [0, 2**40)) so that direct addressing cannot apply;
  * Zipf(s) is truncated to ranks 1..K, P(r) ~ r**-s, sampled by inverse CDF; rank r is mapped to a
    key through a seeded permutation so the hot keys are scattered over the key space;
  * "N(0, v)" means variance v.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Relations", "Branch", "rng_for", "draw_keys", "zipf_ranks", "draw_tuples", "make_rule",
    "config1", "config2", "config3", "config4", "serving_trace", "serving_query",
]


def rng_for(seed: int, *stream: int) -> np.random.Generator:
    """Independent PCG64 stream for (seed, *stream)."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, *stream])))


def draw_keys(rng: np.random.Generator, k: int, key_dtype=np.int32, sparse: bool = False) -> np.ndarray:
    """K distinct keys in shuffled order (the H.id column)."""
    if sparse:
        hi = (1 << 40) if np.dtype(key_dtype) == np.int64 else (1 << 30)
        vals = np.unique(rng.integers(0, hi, size=int(k * 1.05) + 16, dtype=np.int64))
        while vals.size < k:
            vals = np.unique(np.concatenate([vals, rng.integers(0, hi, size=k, dtype=np.int64)]))
        vals = rng.permutation(vals)[:k]
        return vals.astype(key_dtype)
    return rng.permutation(k).astype(key_dtype)


def zipf_ranks(rng: np.random.Generator, n: int, k: int, s: float) -> np.ndarray:
    """n draws of ranks 0..k-1 with P(rank r) proportional to (r+1)**-s (truncated Zipf)."""
    w = np.arange(1, k + 1, dtype=np.float64) ** (-float(s))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    u = rng.random(n)
    r = np.searchsorted(cdf, u, side="right")
    return np.minimum(r, k - 1).astype(np.int64)


def draw_tuples(rng: np.random.Generator, n: int, keys: np.ndarray, dist: str = "uniform",
                s: float = 1.0) -> np.ndarray:
    """n key values drawn from ``keys`` either uniformly or by truncated Zipf(s) over a seeded
    permutation of the keys."""
    k = keys.size
    if dist == "uniform":
        idx = rng.integers(0, k, size=n)
    elif dist == "zipf":
        perm = rng.permutation(k)
        idx = perm[zipf_ranks(rng, n, k, s)]
    else:
        raise ValueError(dist)
    return keys[idx]


@dataclasses.dataclass
class Branch:
    """One tuple relation E(src, dst [; r]) with its own Linear(W, b)."""
    src: np.ndarray
    dst: np.ndarray
    W: np.ndarray | None          # [d_out, d_in] float32 (torch nn.Linear layout), None = identity
    b: np.ndarray | None          # [d_out] float32
    r: np.ndarray | None = None   # [T, d_r] float32 per-tuple embedding, or None


@dataclasses.dataclass
class Relations:
    """H(id; z) plus one or more branches E_i; embeddings are float32 on the host."""
    h_ids: np.ndarray
    z: np.ndarray
    branches: list
    act: str = "none"
    join_dst: bool = True
    concat_dst: bool = True


def _normal(rng, shape, var):
    return (rng.standard_normal(shape) * math.sqrt(var)).astype(np.float32)


def make_rule(seed: int, n_tuples: int, n_keys: int, d: int, d_out: int, key_dtype=np.int32,
              src_dist: str = "uniform", src_s: float = 1.0, dst_dist: str = "uniform",
              dst_s: float = 1.0, d_r: int = 0, act: str = "none", n_branches: int = 1,
              branch_tuples=None, sparse_keys: bool = False, w_var: float | None = None,
              missing_frac: float = 0.0, dup_frac: float = 0.0) -> Relations:
    """A rule instance H'(dst; SUM Linear(Concat(z_src, z_dst[, r]))) over synthetic relations.

    ``missing_frac``: fraction of E keys replaced by keys absent from H (dropped by the join).
    ``dup_frac``: fraction of H rows duplicated with a fresh embedding (bag semantics on H)."""
    rng = rng_for(seed, 1)
    keys = draw_keys(rng, n_keys, key_dtype, sparse_keys)
    h_ids = keys.copy()
    z = _normal(rng, (n_keys, d), 1.0)
    if dup_frac > 0:
        nd = max(1, int(n_keys * dup_frac))
        pick = rng.integers(0, n_keys, size=nd)
        h_ids = np.concatenate([h_ids, keys[pick]])
        z = np.concatenate([z, _normal(rng, (nd, d), 1.0)])
        perm = rng.permutation(h_ids.size)
        h_ids, z = h_ids[perm], z[perm]
    d_in = 2 * d + d_r
    var = (1.0 / d_in) if w_var is None else w_var
    sizes = branch_tuples if branch_tuples is not None else [n_tuples] * n_branches
    branches = []
    for i, t in enumerate(sizes):
        brng = rng_for(seed, 2, i)
        src = draw_tuples(brng, t, keys, src_dist, src_s)
        dst = draw_tuples(brng, t, keys, dst_dist, dst_s)
        if missing_frac > 0:
            big = np.int64(keys.max()) + 1
            for col in (src, dst):
                m = brng.random(t) < missing_frac
                col[m] = (big + brng.integers(0, 1000, size=int(m.sum()))).astype(col.dtype)
        W = _normal(brng, (d_out, d_in), var)
        b = _normal(brng, (d_out,), var)
        r = _normal(brng, (t, d_r), 1.0) if d_r > 0 else None
        branches.append(Branch(src=src.astype(key_dtype), dst=dst.astype(key_dtype), W=W, b=b, r=r))
    return Relations(h_ids=h_ids.astype(key_dtype), z=z, branches=branches, act=act)


def config1(seed: int = 0) -> Relations:
    """Plain single rule, FP32 form: E 2,000 tuples, src/dst uniform over 500 int32 keys,
    z f32[16] ~ N(0,1), W 16x32 and b[16] ~ N(0, 1/32)."""
    return make_rule(seed, 2000, 500, 16, 16, np.int32, w_var=1.0 / 32)


def config2(seed: int = 0, n_tuples: int = 16_000_000, n_keys: int = 1_000_000) -> Relations:
    """Single rule at scale: E 16M tuples over 1M int64 keys, src ~ Zipf(1.1), dst uniform,
    z[128] ~ N(0,1) (the device copy is bf16), W 128x256, b[128] ~ N(0, 1/256)."""
    return make_rule(seed, n_tuples, n_keys, 128, 128, np.int64, src_dist="zipf", src_s=1.1)


def config3(seed: int = 0, n_tuples: int = 4_000_000, n_keys: int = 500_000):
    """Two stacked rules plus a SUM readout: E 4M tuples over 500k int32 keys, src ~ Zipf(1.2),
    dst uniform, z f32[64]; rule 1 Linear 128->64 + ReLU, rule 2 Linear 128->64; readout into 8
    groups (one uniform group id per key); MSE against N(0,1) targets [8, 64].

    Returns (rule1 Relations, W2, b2, group_ids [n_keys] aligned with h_ids, targets [8,64])."""
    r1 = make_rule(seed, n_tuples, n_keys, 64, 64, np.int32, src_dist="zipf", src_s=1.2,
                   act="relu")
    rng = rng_for(seed, 3)
    W2 = _normal(rng, (64, 128), 1.0 / 128)
    b2 = _normal(rng, (64,), 1.0 / 128)
    groups = rng.integers(0, 8, size=n_keys).astype(np.int32)
    targets = _normal(rng, (8, 64), 1.0)
    return r1, W2, b2, groups, targets


def config4(seed: int = 0, sizes=(2_000_000, 1_000_000, 500_000), n_keys: int = 300_000) -> Relations:
    """Union replicator over 3 relations sharing a 300k int32 key space: src uniform, dst ~
    Zipf(1.0), z f32[64], r_edge f32[64] per tuple, one Linear 192->96 per branch."""
    return make_rule(seed, 0, n_keys, 64, 96, np.int32, dst_dist="zipf", dst_s=1.0, d_r=64,
                     branch_tuples=list(sizes))


def serving_trace(seed: int = 0, n_queries: int = 10_000, rate: float = 2000.0,
                  t_min: int = 1000, t_max: int = 1_000_000):
    """Poisson arrivals (exponential gaps at ``rate``/s) and log-uniform tuple counts."""
    rng = rng_for(seed, 5)
    gaps = rng.exponential(1.0 / rate, size=n_queries)
    arrivals = np.cumsum(gaps) - gaps[0]
    sizes = np.exp(rng.uniform(math.log(t_min), math.log(t_max), size=n_queries)).astype(np.int64)
    return arrivals, sizes


def serving_query(seed: int, q: int, n_tuples: int, d: int = 64):
    """One served query: keys = tuples/8 (at least 1), src/dst uniform, z[64] ~ N(0,1)."""
    rng = rng_for(seed, 6, q)
    k = max(1, int(n_tuples) // 8)
    keys = draw_keys(rng, k, np.int32)
    src = draw_tuples(rng, int(n_tuples), keys)
    dst = draw_tuples(rng, int(n_tuples), keys)
    z = _normal(rng, (k, d), 1.0)
    return keys, src, dst, z


def graph_batch(seed: int, n_graphs: int, n_nodes: int, d: int, near: int = 3, p_back: float = 0.5,
                key_dtype=np.int32, dup_edges: float = 0.0, dup_rows: float = 0.0, missing: float = 0.0):
    """A batch of small directed graphs for the cyclic (triangle) join: graph g's node i has key
    g * n_nodes + i (keys in shuffled H order); every node points to its next `near` nodes on a ring
    and each such edge is also present reversed with probability p_back, so short cycles close.
    ``dup_edges`` repeats a fraction of the edges (bag semantics), ``dup_rows`` repeats H rows with
    fresh embeddings, ``missing`` points a fraction of the edges at keys outside H. Returns
    (h_ids, a, b, c, src, dst) with a, b, c f32 [n_h, d] (N(0, 1))."""
    rng = rng_for(seed, 7)
    g = np.repeat(np.arange(n_graphs, dtype=np.int64), n_nodes * near)
    i = np.tile(np.repeat(np.arange(n_nodes, dtype=np.int64), near), n_graphs)
    k = np.tile(np.arange(1, near + 1, dtype=np.int64), n_graphs * n_nodes)
    j = (i + k) % n_nodes
    src, dst = g * n_nodes + i, g * n_nodes + j
    back = rng.random(src.size) < p_back
    src = np.concatenate([src, dst[back]])
    dst = np.concatenate([dst, (g * n_nodes + i)[back]])
    if dup_edges > 0:
        pick = rng.integers(0, src.size, size=int(src.size * dup_edges))
        src, dst = np.concatenate([src, src[pick]]), np.concatenate([dst, dst[pick]])
    if missing > 0:
        m = rng.random(src.size) < missing
        dst[m] = n_graphs * n_nodes + rng.integers(0, 1000, size=int(m.sum()))
    perm = rng.permutation(src.size)
    src, dst = src[perm], dst[perm]
    h_ids = np.arange(n_graphs * n_nodes, dtype=np.int64)
    if dup_rows > 0:
        h_ids = np.concatenate([h_ids, rng.integers(0, h_ids.size, size=int(h_ids.size * dup_rows))])
    h_ids = h_ids[rng.permutation(h_ids.size)]
    a, b, c = (_normal(rng, (h_ids.size, d), 1.0) for _ in range(3))
    return (h_ids.astype(key_dtype), a, b, c, src.astype(key_dtype), dst.astype(key_dtype))
