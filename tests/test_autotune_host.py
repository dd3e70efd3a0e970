"""Host-side logic of the autotuner (no GPU): the candidate grid, the size buckets, and apply()
setting the library's process-wide knobs (relnn_tune_set runs on the host) and returning the form's
flags."""
import pytest

from paper_2605_24207_b300 import autotune as A
from paper_2605_24207_b300 import relnn as R


def test_candidates_cover_forms_and_defaults():
    c = A.candidates(kahan=False)
    assert dict(A.DEFAULTS) in c
    assert {x["form"] for x in c} == {"agg", "per_tuple", "pushdown"}
    assert {x["agg_epi"] for x in c} == {4, 8}
    assert all(x["kahan_min"] == 33 for x in c)
    assert {x["kahan_min"] for x in A.candidates(kahan=True)} == {0, 33}
    assert {x["agg_fuse"] for x in c} == {0, 1}


def test_size_buckets_are_powers_of_four():
    assert A.size_bucket(1000) == A.size_bucket(4000) - 1 == 4
    assert A.size_bucket(16_000_000) == 11
    assert A.size_bucket(0) == 0


def test_apply_sets_knobs_and_returns_flags():
    saved = {k: R.tune_get(k) for k in range(7)}
    try:
        assert A.apply(dict(form="per_tuple", agg_rows=32, agg_stages=3, agg_epi=4, kahan_min=17,
                            sort_bits=10, group_sort=1)) == R.FLAG_PER_TUPLE
        assert [R.tune_get(k) for k in (R.TUNE_AGG_ROWS, R.TUNE_AGG_STAGES, R.TUNE_AGG_EPI, R.TUNE_KAHAN_MIN,
                                        R.TUNE_SORT_BITS, R.TUNE_GROUP_SORT)] == [32, 3, 4, 17, 10, 1]
        assert A.apply(dict(form="per_tuple", tile128=True)) == R.FLAG_PER_TUPLE | R.FLAG_TILE128
        assert A.apply({"form": "pushdown"}) == R.FLAG_PUSHDOWN
        assert R.tune_get(R.TUNE_AGG_EPI) == 8 and R.tune_get(R.TUNE_SORT_BITS) == 8
        assert R.tune_get(R.TUNE_GROUP_SORT) == 0
        assert A.apply(None) == 0
        with pytest.raises(R.RelnnError):
            R.tune_set(R.TUNE_AGG_EPI, 6)
        with pytest.raises(R.RelnnError):
            R.tune_set(R.TUNE_AGG_STAGES, 1)
    finally:
        for k, v in saved.items():
            R.tune_set(k, v)
