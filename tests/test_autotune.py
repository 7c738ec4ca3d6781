"""The autotuner's layout signature and its cache (host logic, no GPU)."""
import json

from paper_2605_14277_b300 import autotune as A
from paper_2605_14277_b300 import games as G


def test_signature_groups_loads_of_the_same_kind():
    a = G.batch_games(64)
    b = [G.batch_game(s) for s in G.batch_sample_seeds(64)]
    assert A.signature(a) == A.signature(a[::-1])        # order does not matter
    assert A.signature(a, "cfr+") != A.signature(a, "dcfr")
    assert A.signature(a, iterations=64) != A.signature(a, iterations=8)
    assert A.signature(a[:8]) != A.signature(a)          # 8 games vs 64
    assert A.signature(G.rps()) != A.signature(G.poker_game())
    assert isinstance(A.signature(b), str)


def test_cached_choice_is_returned_without_timing(tmp_path):
    trees = G.batch_games(16)
    path = tmp_path / "tune.json"
    key = A.signature(trees, "cfr+", 64)
    entry = {"shape": 3, "flat": True, "passes": 1, "us_per_iteration": 12.5,
             "table": [[3, True, 1, 12.5], [2, False, 1, 14.0]]}
    path.write_text(json.dumps({key: entry, "other": {"shape": 1}}))
    # a cache hit never loads a solver (there is no GPU here)
    got = A.tune(trees, "cfr+", iterations=64, cache=str(path))
    assert got["cached"] and got["signature"] == key
    assert (got["shape"], got["flat"], got["passes"]) == (3, True, 1)
    assert got["table"][1] == (2, False, 1, 14.0)


def test_cache_put_keeps_other_entries(tmp_path):
    path = str(tmp_path / "tune.json")
    A._cache_put(path, "a", {"shape": 1})
    A._cache_put(path, "b", {"shape": 2})
    A._cache_put(path, "a", {"shape": 4})
    data = json.loads(open(path).read())
    assert data == {"a": {"shape": 4}, "b": {"shape": 2}}
