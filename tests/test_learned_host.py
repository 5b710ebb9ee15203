"""Host-side pieces of the learned-proposal pipeline."""
import numpy as np

from paper_2511_20317_gb300 import learned, tfg


def test_canonical_order_is_independent_of_arrival_order():
    rng = np.random.default_rng(0)
    e = np.zeros(500, dtype=tfg.LOG_ENTRY_DTYPE)
    e["walker_id"] = rng.integers(0, 20, 500)
    e["step"] = rng.integers(0, 50, 500)
    e["label"] = rng.integers(0, 2, 500)
    e["feat"] = rng.integers(0, 2**16, (500, 32))
    a = learned.canonical_order(e)
    b = learned.canonical_order(e[rng.permutation(500)])
    key = lambda x: np.stack([x["walker_id"], x["step"], x["label"].astype(np.int64)], 1)
    assert np.array_equal(key(a), key(b))
    k = key(a)
    assert (np.diff(k[:, 0]) >= 0).all()
    same_w = np.diff(k[:, 0]) == 0
    assert (np.diff(k[:, 1])[same_w] >= 0).all()


def run(v, low, hist):
    return {"net_descent": v, "mean_best_rank": 64 - v, "lowest_rank": low, "reductions_per_1e9_applied": 100 * v,
            "steps_per_s": 1e8, "steps_per_walker": 1500, "rank_hist": hist, "verify_failures": 0,
            "collected_verified": True}


def test_summary_intervals_and_the_beats_rule():
    """Means with 95% intervals over the seeds (1.96 s / sqrt(n)); one arm beats
    the other only when the intervals do not overlap; histograms add up."""
    a = learned._summary([run(v, 63, {63: 1, 64: 9}) for v in (3.0, 3.2, 2.8)])
    b = learned._summary([run(v, 63, {63: 2, 64: 8}) for v in (1.0, 1.1, 0.9)])
    c = learned._summary([run(v, 63, {64: 10}) for v in (2.0, 3.5, 0.5)])
    s = np.std([3.0, 3.2, 2.8], ddof=1)
    assert abs(a["net_descent"]["mean"] - 3.0) < 1e-12
    assert abs(a["net_descent"]["ci95"] - 1.96 * s / np.sqrt(3)) < 1e-12
    assert a["rank_hist_all_seeds"] == {63: 3, 64: 27}
    assert learned._beats(a, b, "net_descent") and not learned._beats(b, a, "net_descent")
    assert not learned._beats(c, b, "net_descent")           # overlapping intervals
    assert learned._beats(b, a, "mean_best_rank", higher_better=False) is False
    assert learned._beats(a, b, "mean_best_rank", higher_better=False)
