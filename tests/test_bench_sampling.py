"""The batched benchmark's stratified sample (bench.py, host logic): one
random-walk and one ECG-like query per length x window-ratio stratum of the
1,024-query mix, and the per-(stratum, kind) counts that weight the full-mix
estimate."""
import bench


def test_mix_is_reproducible_and_in_range():
    a = bench.batched_mix(bench.BATCH_FULL_QUERIES)
    b = bench.batched_mix(bench.BATCH_FULL_QUERIES)
    assert a == b and len(a) == 1024
    for m, w, ecg, k, ratio in a:
        assert 64 <= m <= 2048 and 0 <= w <= m and k in (1, 5) and 0.0 <= ratio < 1.0
        assert 0 <= bench._stratum(m, ratio) < 16


def test_sample_takes_the_first_query_of_each_stratum_and_kind():
    mix = bench.batched_mix(bench.BATCH_FULL_QUERIES)
    picked, counts = bench.sample_strata(mix, 32)
    assert sum(counts.values()) == len(mix)   # the weights cover the whole mix
    assert len(picked) == len(counts) == len(set(picked))
    keys = [(bench._stratum(mix[q][0], mix[q][4]), bool(mix[q][2])) for q in picked]
    assert len(set(keys)) == len(keys) == len(counts)
    for q, key in zip(picked, keys):   # no earlier query of the mix has the same (stratum, kind)
        assert all((bench._stratum(m, r), bool(e)) != key for m, w, e, k, r in mix[:q])
    # both kinds of series in every stratum the mix populates
    strata = {s for s, _ in counts}
    assert all((s, True) in counts and (s, False) in counts for s in strata)
    assert bench.sample_strata(mix, 5)[0] == picked[:5]
