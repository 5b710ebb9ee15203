"""Tensor-core MLP of the learned proposal against the float64 reference."""
import numpy as np
import pytest

from oracle import mlp
from paper_2511_20317_gb300 import tfg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def gpu():
    import torch
    assert torch.cuda.is_available()
    from paper_2511_20317_gb300 import _build
    _build.build()
    tfg.lib()


def device_params(p):
    import torch
    blob = np.frombuffer(p.blob(), dtype=np.uint8)
    assert blob.size == tfg.tfg_mlp_param_bytes()
    return torch.from_numpy(blob.copy()).cuda()


def device_rows(x):
    import torch
    bits = mlp.bf16_bits(mlp.bf16_round(x))
    return torch.from_numpy(bits.view(np.int16).copy()).cuda().view(torch.bfloat16)


@pytest.mark.parametrize("n", [1, 127, 128, 1000, 128 * 700 + 5])
def test_score_matches_reference(n):
    rng = np.random.default_rng(n)
    p = mlp.Params.random(rng)
    x = rng.integers(0, 9, size=(n, mlp.IN)).astype(np.float32)
    x[:, 20:] = rng.normal(0, 2, size=(n, mlp.IN - 20))
    want, cache = mlp.forward(p, x)
    got = tfg.tfg_mlp_score(device_params(p), device_rows(x)).cpu().numpy().astype(np.float64)
    # The device accumulates in FP32, the reference in FP64; where a first-layer
    # unit lands within that difference of a bf16 rounding midpoint the two round
    # it one bf16 ulp (2^-8 relative) apart.  Bound: two such flips per row, each
    # moving the score by at most ulp(h1_h) * sum_o |W2[h,o] w3[o]|, plus FP32
    # accumulation error of the two products.
    h1 = cache[2]
    path = np.abs(p.W2) @ np.abs(p.w3)                      # per hidden unit
    flip = (np.abs(h1) * 2.0 ** -8) * path                   # [n, 128]
    bound = 2 * flip.max(axis=1) + 1e-5 * (1 + np.abs(want))
    assert (np.abs(got - want) <= bound).all(), np.max(np.abs(got - want) - bound)
    # ranking of candidates (what the proposal uses) agrees except near ties
    if n >= 128:
        order_gap = np.sort(want)[-1] - np.sort(want)[-2]
        if order_gap > 2 * bound.max():
            assert np.argmax(got) == np.argmax(want)


def test_gradients_match_reference():
    """Fused tensor-core forward/backward against the float64 reference with the
    same bf16 operand roundings.  Per-entry bound: one bf16 ulp (2^-8) on each
    operand of every product term, i.e. 2^-7 * sum_s |a_s b_s|, plus FP32 sum error."""
    import torch
    rng = np.random.default_rng(7)
    p = mlp.Params.random(rng)
    n = 128 * 300 + 37
    x = rng.integers(0, 9, size=(n, mlp.IN)).astype(np.float32)
    x[:, 24:] = mlp.bf16_round(rng.normal(0, 1, size=(n, mlp.IN - 24)))
    label = (rng.random(n) < 0.3).astype(np.float32)
    weight = np.where(label > 0, 0.5 / max(label.sum(), 1), 0.5 / max((1 - label).sum(), 1)).astype(np.float32)
    y, cache = mlp.forward(p, x)
    loss, dy = mlp.logistic_loss(y, label, weight)
    ref = mlp.backward(p, cache, dy, bf16_operands=True)
    g, gloss = tfg.tfg_mlp_grad(device_params(p), device_rows(x), torch.from_numpy(label).cuda(),
                                torch.from_numpy(weight).cuda())
    got = mlp.split_vector(g.cpu().numpy().astype(np.float64))
    assert abs(gloss - loss) <= 1e-4 * (1 + abs(loss))
    for name in ["W1", "W2", "b1", "b2", "w3", "b3"]:
        bound = 2.0 ** -7 * np.asarray(ref["_abs"][name]) + 1e-6 * (1 + np.abs(ref[name]))
        diff = np.abs(np.asarray(got[name]) - np.asarray(ref[name]))
        assert (diff <= bound).all(), (name, float(np.max(diff - bound)))


def test_training_learns_a_separable_rule():
    """Adam steps on the device drive the loss of a learnable labelling down."""
    import torch
    rng = np.random.default_rng(3)
    p = mlp.Params.random(rng, scale=0.5)
    n = 128 * 64
    x = rng.integers(0, 9, size=(n, mlp.IN)).astype(np.float32)
    label = ((x[:, 0] + x[:, 3] - x[:, 5]) > 5).astype(np.float32)
    weight = np.full(n, 1.0 / n, np.float32)
    params = device_params(p)
    xs, ls, ws = device_rows(x), torch.from_numpy(label).cuda(), torch.from_numpy(weight).cuda()
    tr = tfg.MlpTrainer(params)
    _, loss0 = tfg.tfg_mlp_grad(params, xs, ls, ws)
    for _ in range(300):
        tr.step(xs, ls, ws, 3e-3)
    _, loss1 = tfg.tfg_mlp_grad(params, xs, ls, ws)
    assert loss1 < 0.5 * loss0, (loss0, loss1)
    acc = ((tfg.tfg_mlp_score(params, xs).cpu().numpy() > 0) == (label > 0)).mean()
    assert acc > 0.9, acc


def test_adam_step_matches_reference_elementwise():
    """Six device training steps against the float64 Adam of the reference fed
    with the device's own gradient of each step: FP32 master weights, both
    moments and the parameter blob (bf16 W1, W2 = the rounded master weights,
    the rest the FP32 master values) element by element.  Bound: FP32 rounding
    of each update (a few 2^-24 relative of the moment and update terms) per
    step, accumulated over the steps."""
    import torch
    rng = np.random.default_rng(12)
    p = mlp.Params.random(rng)
    n = 128 * 40 + 9
    x = rng.integers(0, 9, size=(n, mlp.IN)).astype(np.float32)
    label = (rng.random(n) < 0.3).astype(np.float32)
    weight = np.full(n, 1.0 / n, np.float32)
    params = device_params(p)
    xs, ls, ws = device_rows(x), torch.from_numpy(label).cuda(), torch.from_numpy(weight).cuda()
    tr = tfg.MlpTrainer(params)
    P = mlp.NUM_PARAMS
    state = lambda k: tr.state[k * P:(k + 1) * P].cpu().numpy().astype(np.float64)
    opt = mlp.Adam(state(0))
    assert (opt.m == 0).all() and np.array_equal(state(1), np.zeros(P)) and np.array_equal(state(2), np.zeros(P))
    lr, steps, gmax = 2e-3, 6, 0.0
    for k in range(1, steps + 1):
        tr.step(xs, ls, ws, lr)
        g = state(3)                      # the gradient this step used
        gmax = max(gmax, float(np.abs(g).max()))
        opt.step(g, lr)
    tol = 2.0 ** -21 * steps
    assert (np.abs(state(1) - opt.m) <= tol * (np.abs(opt.m) + gmax * 1e-3)).all()
    assert (np.abs(state(2) - opt.v) <= tol * (np.abs(opt.v) + gmax ** 2 * 1e-6)).all()
    master = state(0)
    assert (np.abs(master - opt.theta) <= tol * (np.abs(opt.theta) + lr)).all(), \
        float(np.max(np.abs(master - opt.theta)))
    # the blob: bf16 of the FP32 master for W1, W2; the FP32 master values for the rest
    blob = params.cpu().numpy()
    nw = mlp.IN * mlp.HID + mlp.HID * mlp.HID
    m32 = tr.state[:P].cpu().numpy()
    assert np.array_equal(blob[:2 * nw].view(np.uint16), mlp.bf16_bits(mlp.bf16_round(m32[:nw])))
    assert np.array_equal(blob[2 * nw:2 * nw + 4 * (P - nw)].view(np.float32), m32[nw:])


def test_training_steps_are_bit_reproducible():
    """The training step adds the per-CTA gradient rows in CTA order (no
    floating-point atomics): two trainers started from the same parameters on
    the same batches end with the same bits, and their gradients equal the
    atomic-sum gradient of tfg_mlp_grad to rounding."""
    import torch
    rng = np.random.default_rng(5)
    p = mlp.Params.random(rng, scale=0.5)
    n = 128 * 300 + 17                      # more tiles than SMs, a ragged last tile
    x = rng.integers(0, 9, size=(n, mlp.IN)).astype(np.float32)
    label = (rng.random(n) < 0.3).astype(np.float32)
    weight = np.full(n, 1.0 / n, np.float32)
    xs, ls, ws = device_rows(x), torch.from_numpy(label).cuda(), torch.from_numpy(weight).cuda()
    blobs, states = [], []
    for _ in range(2):
        params = device_params(p)
        tr = tfg.MlpTrainer(params)
        for _ in range(5):
            tr.step(xs, ls, ws, 3e-3)
        torch.cuda.synchronize()
        blobs.append(params.cpu().numpy())
        states.append(tr.state[: 4 * tfg.MLP_NUM_PARAMS + 1].cpu().numpy())
    assert np.array_equal(blobs[0], blobs[1])
    assert np.array_equal(states[0].view(np.uint32), states[1].view(np.uint32))
    # the ordered gradient against the atomic-sum gradient at the same parameters
    params = device_params(p)
    tr = tfg.MlpTrainer(params)
    tr.step(xs, ls, ws, 0.0)                 # lr 0: the parameters stay, the gradient is kept
    g_det = tr.state[3 * tfg.MLP_NUM_PARAMS: 4 * tfg.MLP_NUM_PARAMS].cpu().numpy().astype(np.float64)
    g_atom, _ = tfg.tfg_mlp_grad(params, xs, ls, ws)
    g_atom = g_atom.cpu().numpy().astype(np.float64)
    assert np.allclose(g_det, g_atom, rtol=1e-4, atol=1e-7 * np.abs(g_atom).max())
