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
