"""The allocation-free window-mode entry point (tfg_walk_window_noalloc).

It serves callers that cannot call cudaMalloc: its per-step scratch is the
library's own static device array.  Its results must equal those of the
entry point that takes caller scratch, call after call: the array is shared
and keeps the previous call's contents, which the step must never read.
Collected last so that a failure here stops a -x run only after every other
test has run."""
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


def test_noalloc_equals_caller_scratch_entry_point_two_calls():
    import torch
    fmt, nw, steps, seed = (3, 3, 3), 1500, 120, 21
    start = naive_start(*fmt)
    blob = np.frombuffer(mlp.Params.random(np.random.default_rng(5)).blob(), dtype=np.uint8).copy()
    params = torch.from_numpy(blob).cuda()
    eps = int(0.2 * 2**32)
    p = tfg.tfg_default_params(plateau_len=60)
    A = tfg.Walkers([(fmt, 0, start, nw)], seed=seed, params=p)
    B = tfg.Walkers([(fmt, 0, start, nw)], seed=seed, params=p)
    for call in range(2):
        ca = A.walk_window(steps, policy=1, mlp_params=params, eps_thresh=eps, record_choices=True)
        cb = torch.full((steps, nw), -2, dtype=torch.int32, device="cuda")
        B.walk_window_noalloc(steps, policy=1, mlp_params=params, eps_thresh=eps, d_choices=cb)
        B.sync()
        # the walk is integer arithmetic and the network is deterministic: equality
        assert torch.equal(ca, cb), f"call {call}: chosen candidates differ"
        ia, sa, ba = A.read_walkers(0, nw)
        ib, sb, bb = B.read_walkers(0, nw)
        assert np.array_equal(ia, ib) and np.array_equal(sa, sb) and np.array_equal(ba, bb), f"call {call}"
    assert B.verify_all() == 0
    st, _ = B.stats()
    assert st["steps"] == 2 * steps * nw and st["reductions"] > 0


def test_noalloc_calls_leave_free_device_memory_unchanged():
    """After one warm-up call (which loads the kernels' modules), further calls
    take no device memory: the free bytes the driver reports stay the same."""
    import torch
    fmt, nw = (3, 3, 3), 1000
    start = naive_start(*fmt)
    params = torch.from_numpy(np.frombuffer(mlp.Params.random(np.random.default_rng(8)).blob(),
                                            dtype=np.uint8).copy()).cuda()
    W = tfg.Walkers([(fmt, 0, start, nw)], seed=2, params=tfg.tfg_default_params(plateau_len=60))
    ch = torch.full((4, nw), -2, dtype=torch.int32, device="cuda")
    W.walk_window_noalloc(1, policy=1, mlp_params=params, eps_thresh=int(0.1 * 2**32))
    W.sync()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        W.walk_window_noalloc(4, policy=1, mlp_params=params, eps_thresh=int(0.1 * 2**32), d_choices=ch)
        W.sync()
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
    assert (ch >= -1).all()


def test_noalloc_rejects_a_context_of_another_device():
    import torch
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two devices")
    fmt = (2, 2, 2)
    with torch.cuda.device(1):
        W = tfg.Walkers([(fmt, 0, naive_start(*fmt), 64)], seed=1)
    with torch.cuda.device(0):
        with pytest.raises(tfg.TfgError) as e:
            W.walk_window_noalloc(1, policy=0)
    assert e.value.code == tfg.TFG_EINVAL and "current" in str(e.value)


def test_noalloc_rejects_contexts_beyond_the_static_capacity():
    fmt = (2, 2, 2)
    W = tfg.Walkers([(fmt, 0, naive_start(*fmt), 20000)], seed=1)
    with pytest.raises(tfg.TfgError) as e:
        W.walk_window_noalloc(1, policy=0)
    assert e.value.code == tfg.TFG_EINVAL and "static scratch" in str(e.value)
