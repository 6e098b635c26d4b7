"""The autotuner's search logic on CPU with a synthetic cost: coordinate
search over the candidate lists, the noise margin, failed checks, and the
JSON store."""
from paper_2001_11619_gb300 import autotune as A


def _cost(cfg):
    # separable cost with a known minimum at (128, 40, 8)
    ms = 100.0
    ms += abs(cfg["cluster_min_n"] - 128) * 0.05
    ms += abs(cfg["cluster_level_boxes"] - 40) * 0.02
    ms += {4: 3.0, 8: 0.0, 16: 1.0}[cfg["sweep_rhs_chunk"]]
    return ms


START = {"cluster_min_n": 160, "cluster_level_boxes": 76, "sweep_rhs_chunk": 16}
CAND = {k: A.CANDIDATES[k] for k in START}


def test_search_finds_the_separable_minimum():
    calls = []

    def measure(cfg):
        calls.append(dict(cfg))
        return _cost(cfg), True

    best, ms, log = A.search(measure, START, CAND, noise=0.0)
    assert best == {"cluster_min_n": 128, "cluster_level_boxes": 40,
                    "sweep_rhs_chunk": 8}
    assert ms == _cost(best)
    # one measurement of the start, then each other candidate once
    n = 1 + sum(len(vals) - 1 for vals in CAND.values())
    assert len(calls) == n == len(log)


def test_noise_margin_and_failed_checks():
    def measure(cfg):
        ms = _cost(cfg)
        # the fastest sweep chunk fails its accuracy check
        return ms, cfg["sweep_rhs_chunk"] != 8

    best, ms, log = A.search(measure, START, CAND, noise=0.0)
    assert best["sweep_rhs_chunk"] == 16
    assert any(not ok for _, _, ok in log)
    # a large noise margin keeps the start: no change is clearly faster
    best, ms, _ = A.search(lambda c: (_cost(c), True), START, CAND, noise=0.5)
    assert best == START


def test_store_round_trip(tmp_path):
    p = str(tmp_path / "tune.json")
    assert A.load(p, "k") is None
    A.save(p, "k", {"config": START, "ms": 1.0, "default_ms": 2.0})
    A.save(p, "k2", {"config": {"sweep_rhs_chunk": 4}, "ms": 1.0,
                     "default_ms": 1.0})
    assert A.load(p, "k") == START
    assert A.load(p, "k2") == {"sweep_rhs_chunk": 4}
