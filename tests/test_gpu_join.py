"""GPU parity of relnn_join_build / relnn_join_probe against the FP64 oracle's join (bit-exact,
same order: probe row, then build row)."""
import numpy as np
import pytest
import torch

from oracle import relnn_oracle as O
from paper_2605_24207_b300 import relnn as R

pytestmark = pytest.mark.gpu


def _case(seed, n_build, n_probe, key_dtype, span, dup=True, neg=False):
    rng = np.random.default_rng(seed)
    lo = -span if neg else 0
    build = rng.integers(lo, span, size=n_build).astype(key_dtype)
    if not dup:  # distinct keys drawn from a possibly huge range
        u = np.unique(rng.integers(lo, span, size=2 * n_build))
        build = rng.permutation(u)[:n_build].astype(key_dtype)
    probe = rng.integers(lo - 5, span + 5, size=n_probe).astype(key_dtype)
    return build, probe


@pytest.mark.parametrize("key_dtype", [np.int32, np.int64])
@pytest.mark.parametrize("span,dup,neg", [(3000, True, False), (1 << 40, False, False), (2000, True, True),
                                          (50_000, False, True)])
def test_probe_matches_oracle(gpu, key_dtype, span, dup, neg):
    if key_dtype == np.int32 and span > (1 << 30):
        span = (1 << 30)
    build, probe = _case(1, 5000, 20_011, key_dtype, span, dup, neg)
    j = R.Join(torch.from_numpy(build).cuda())
    pi, bi = j.probe(torch.from_numpy(probe).cuda())
    opi, obi = O.join_pairs(probe, build)
    assert np.array_equal(pi.cpu().numpy(), opi)
    assert np.array_equal(bi.cpu().numpy(), obi)


def test_probe_enospc_reports_required_size(gpu):
    build = np.array([1, 1, 1, 2], np.int32)
    probe = np.array([1, 2, 3, 1], np.int32)
    j = R.Join(torch.from_numpy(build).cuda())
    with pytest.raises(R.RelnnError) as e:
        j.probe(torch.from_numpy(probe).cuda(), capacity=3)
    assert e.value.status == 3
    pi, bi = j.probe(torch.from_numpy(probe).cuda())
    assert pi.numel() == 7


def test_empty_sides(gpu):
    j = R.Join(torch.zeros(0, dtype=torch.int64, device="cuda"))
    pi, bi = j.probe(torch.arange(10, dtype=torch.int64, device="cuda"))
    assert pi.numel() == 0
    j2 = R.Join(torch.arange(10, dtype=torch.int64, device="cuda"))
    pi, bi = j2.probe(torch.zeros(0, dtype=torch.int64, device="cuda"))
    assert pi.numel() == 0


def test_reserved_key_rejected(gpu):
    with pytest.raises(R.RelnnError) as e:
        R.Join(torch.tensor([1, np.iinfo(np.int64).max], dtype=torch.int64, device="cuda"))
    assert e.value.status == 1


def test_cardinality_invariant_large(gpu):
    """|P |><| B| = sum_k c_P(k) c_B(k) on 2M probe keys with skewed duplicates."""
    rng = np.random.default_rng(7)
    build = rng.integers(0, 100_000, size=300_000).astype(np.int64)
    probe = (rng.zipf(1.3, size=2_000_000) % 120_000).astype(np.int64)
    j = R.Join(torch.from_numpy(build).cuda())
    pi, bi = j.probe(torch.from_numpy(probe).cuda())
    cb = np.bincount(build, minlength=200_000)
    cp = np.bincount(probe, minlength=200_000)
    assert pi.numel() == int(np.sum(cb.astype(np.int64) * cp))
    # every emitted pair is a real match, in (probe, build) order
    p, b = pi.cpu().numpy(), bi.cpu().numpy()
    assert np.all(probe[p] == build[b])
    order = p.astype(np.int64) * 400_000 + b
    assert np.all(np.diff(order) > 0)
