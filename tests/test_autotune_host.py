"""Host logic of the batched-launch autotuner (CPU only): the candidate set,
the choice of the fastest shape, the per-signature cache and its keys.  The
timing callback is a stand-in for the CUDA-event timing of the real calls."""

import json

import pytest

from paper_2404_01407_gb300 import autotune, fnlh


@pytest.fixture()
def cache_file(tmp_path, monkeypatch):
    path = tmp_path / "_build" / "autotune.json"
    monkeypatch.setattr(autotune, "CACHE", str(path))
    return path


def test_candidates_cover_the_search_space_and_the_per_row_mode():
    c = [(t.threads, t.ctas_per_sm) for t in autotune.candidates()]
    shared = [(th, k) for th in autotune.SEARCH_THREADS for k in autotune.SEARCH_CTAS_PER_SM]
    assert c[:-1] == shared
    assert c[-1] == (0, fnlh.FNLH_TUNING_PER_ROW)
    assert len(set(c)) == len(c)


def test_fastest_shape_wins_and_the_table_lists_every_candidate(cache_file):
    def fake_ms(t):  # a unique minimum at 128 threads, 4 CTAs per SM
        return 10.0 + abs(t.threads - 128) / 64 + abs(t.ctas_per_sm - 4)

    best, table = autotune.tune_batched(fake_ms)
    assert (best.threads, best.ctas_per_sm) == (128, 4)
    assert len(table) == len(list(autotune.candidates()))
    assert min(table, key=lambda r: r["ms"]) == {"threads": 128, "ctas_per_sm": 4, "ms": 10.0}
    assert not cache_file.exists()  # no key: nothing cached


def test_ties_keep_the_first_candidate(cache_file):
    best, _ = autotune.tune_batched(lambda t: 1.0)
    first = next(autotune.candidates())
    assert (best.threads, best.ctas_per_sm) == (first.threads, first.ctas_per_sm)


def test_per_row_mode_can_win(cache_file):
    best, _ = autotune.tune_batched(lambda t: 1.0 if t.ctas_per_sm == fnlh.FNLH_TUNING_PER_ROW else 2.0)
    assert best.ctas_per_sm == fnlh.FNLH_TUNING_PER_ROW


def test_cache_per_signature(cache_file):
    calls = []

    def fake_ms(t):
        calls.append((t.threads, t.ctas_per_sm))
        return 5.0 if (t.threads, t.ctas_per_sm) == (64, 0) else 7.0

    key = autotune.signature(6, [3, 9, 5], [200_000, 600_000, 1_100_000], fnlh.FNLH_BF16, 152)
    best, table = autotune.tune_batched(fake_ms, key=key)
    n = len(calls)
    assert n == len(list(autotune.candidates()))
    stored = json.loads(cache_file.read_text())
    assert stored[key]["threads"] == 64 and stored[key]["ctas_per_sm"] == 0 and stored[key]["ms"] == 5.0
    # a second call with the same signature reads the cache and times nothing
    best2, table2 = autotune.tune_batched(fake_ms, key=key)
    assert len(calls) == n
    assert (best2.threads, best2.ctas_per_sm) == (64, 0) and table2 == table
    # use_cache=False re-times and overwrites
    autotune.tune_batched(lambda t: 3.0 if t.threads == 256 and t.ctas_per_sm == 8 else 9.0, key=key,
                          use_cache=False)
    assert json.loads(cache_file.read_text())[key]["threads"] == 256


def test_signature_buckets_node_counts_by_powers_of_two():
    s = autotune.signature
    assert s(6, [9], [600_000], 2, 152) == s(6, [9], [620_000], 2, 152)  # same log2 bucket
    assert s(6, [9], [600_000], 2, 152) != s(6, [9], [1_200_000], 2, 152)
    assert s(6, [9], [600_000], 2, 152) != s(6, [17], [600_000], 2, 152)  # systems per row
    assert s(6, [9], [600_000], 2, 152) != s(6, [9], [600_000], 1, 152)  # precision
    assert s(6, [9], [600_000], 2, 152) != s(6, [9], [600_000], 2, 148)  # SM count
    assert s(5, [3, 9], [0, 1], 2, 152).startswith("b5|K3-9|n0-0|")
