"""Autotuner for the launch shape of the batched persistent sweep.

Searches threads per CTA (= (node, system) pairs per tile) and the grid shape
(one CTA per tile, or a persistent grid of SMs x ctas_per_sm CTAs), and the
per-row mode (every row its own single-row launches: rows that fill the GPU
on their own gain nothing from sharing one), by timing the real calls with
CUDA events, and caches the winner per problem signature (block size,
per-row systems, node-count bucket, precision, SM count) in a JSON file next
to the library (git-ignored).
"""

from __future__ import annotations

import json
import math
import os

from . import fnlh

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")

SEARCH_THREADS = (64, 128, 256)
SEARCH_CTAS_PER_SM = (0, 2, 4, 8)  # 0: one CTA per tile


def signature(block, systems, nodes, precision, sms):
    bucket = [int(round(math.log2(max(n, 1)))) for n in nodes]
    return f"b{block}|K{'-'.join(map(str, systems))}|n{'-'.join(map(str, bucket))}|p{precision}|sm{sms}"


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(cache):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def candidates():
    for th in SEARCH_THREADS:
        for c in SEARCH_CTAS_PER_SM:
            yield fnlh.fnlh_tuning(th, c)
    yield fnlh.fnlh_tuning(0, fnlh.FNLH_TUNING_PER_ROW)


def tune_batched(time_ms, key=None, use_cache=True):
    """time_ms(tuning) -> milliseconds.  Returns (best fnlh_tuning, table)."""
    cache = _load() if (use_cache and key) else {}
    if key and key in cache:
        t = cache[key]
        return fnlh.fnlh_tuning(t["threads"], t["ctas_per_sm"]), cache[key].get("table", [])
    table = []
    best, best_ms = None, float("inf")
    for tn in candidates():
        ms = float(time_ms(tn))
        table.append({"threads": tn.threads, "ctas_per_sm": tn.ctas_per_sm, "ms": ms})
        if ms < best_ms:
            best, best_ms = tn, ms
    if key:
        cache[key] = {"threads": best.threads, "ctas_per_sm": best.ctas_per_sm, "ms": best_ms, "table": table}
        _store(cache)
    return best, table
