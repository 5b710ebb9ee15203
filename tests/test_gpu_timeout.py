"""Bounded device waits report instead of hanging: the scoring network's
first tensor-core completion wait is given a limit of zero polls (the test
hook), so it gives up at once; the kernel then waits, with its normal limit,
for the products in flight, releases its tensor memory and sets its error
word.  In window mode that word is the context's status, which tfg_sync
returns as TFG_ETIMEOUT; the context stays usable and the next call, with the
default limit, runs clean."""
import numpy as np
import pytest

from oracle import mlp
from paper_2511_20317_gb300 import tfg
from paper_2511_20317_gb300.workloads import naive_start

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    assert torch.cuda.is_available()
    from paper_2511_20317_gb300 import _build
    _build.build()
    tfg.lib()
    yield
    tfg.tfg_test_set_wait_limit(-1)


def blob(seed):
    import torch
    return torch.from_numpy(np.frombuffer(mlp.Params.random(np.random.default_rng(seed)).blob(),
                                          dtype=np.uint8).copy()).cuda()


def test_window_step_timeout_returns_etimeout_and_the_context_recovers():
    fmt, nw = (3, 3, 3), 256
    params = blob(2)
    W = tfg.Walkers([(fmt, 0, naive_start(*fmt), nw)], seed=4, params=tfg.tfg_default_params(plateau_len=100))
    W.walk_window(5, policy=1, mlp_params=params, eps_thresh=0)
    W.sync()
    tfg.tfg_test_set_wait_limit(0)
    try:
        W.walk_window(1, policy=1, mlp_params=params, eps_thresh=0)
        with pytest.raises(tfg.TfgError) as e:
            W.sync()
        assert e.value.code == tfg.TFG_ETIMEOUT
    finally:
        tfg.tfg_test_set_wait_limit(-1)
    # read once, cleared after reading
    W.sync()
    W.walk_window(5, policy=1, mlp_params=params, eps_thresh=0)
    W.sync()
    assert W.verify_all() == 0
    st, _ = W.stats()
    assert st["steps"] == 11 * nw


def test_score_timeout_sets_the_error_word_and_a_clean_launch_follows():
    import torch
    rng = np.random.default_rng(3)
    p = mlp.Params.random(rng)
    params = torch.from_numpy(np.frombuffer(p.blob(), dtype=np.uint8).copy()).cuda()
    x = rng.integers(0, 9, size=(1000, mlp.IN)).astype(np.float32)
    xs = torch.from_numpy(mlp.bf16_bits(mlp.bf16_round(x)).view(np.int16).copy()).cuda().view(torch.bfloat16)
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    tfg.tfg_test_set_wait_limit(0)
    try:
        tfg.tfg_mlp_score(params, xs, err=err)
        torch.cuda.synchronize()
        assert int(err.item()) == 1
    finally:
        tfg.tfg_test_set_wait_limit(-1)
    err.zero_()
    got = tfg.tfg_mlp_score(params, xs, err=err).cpu().numpy().astype(np.float64)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    want, cache = mlp.forward(p, x)
    path = np.abs(p.W2) @ np.abs(p.w3)
    bound = 2 * ((np.abs(cache[2]) * 2.0 ** -8) * path).max(axis=1) + 1e-5 * (1 + np.abs(want))
    assert (np.abs(got - want) <= bound).all()
