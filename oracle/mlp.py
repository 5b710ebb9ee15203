"""Reference of the learned flip proposal's network (TEST INFRASTRUCTURE ONLY).

The scoring network 32 -> 128 -> 128 -> 1 with ReLU, written as its plain
definition in numpy float64.  BF16 enters at the points the tensor-core path
fixes: inputs, W1 and W2 are bf16 values, and the first hidden layer is
rounded to bf16 before the second product (round to nearest, ties to even).
Everything else is exact float64 here, so the device path differs only by
FP32 accumulation order (and the rare bf16 rounding flip that causes).
The optimiser of the training step, Adam, is written out as well (class Adam).
"""
from __future__ import annotations

import numpy as np

IN, HID = 32, 128


def bf16_round(x) -> np.ndarray:
    """Round float values to the nearest bf16 (ties to even), returned as float32."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return (r.astype(np.uint32)).view(np.float32)


def bf16_bits(x) -> np.ndarray:
    """bf16 bit patterns (uint16) of values that are already bf16-representable."""
    return (np.asarray(x, dtype=np.float32).view(np.uint32) >> 16).astype(np.uint16)


class Params:
    def __init__(self, W1, b1, W2, b2, w3, b3):
        self.W1 = bf16_round(W1).astype(np.float64)   # [32, 128]
        self.W2 = bf16_round(W2).astype(np.float64)   # [128, 128]
        self.b1 = np.asarray(b1, np.float32).astype(np.float64)
        self.b2 = np.asarray(b2, np.float32).astype(np.float64)
        self.w3 = np.asarray(w3, np.float32).astype(np.float64)
        self.b3 = float(np.float32(b3))

    @staticmethod
    def random(rng, scale=1.0):
        return Params(rng.normal(0, scale / np.sqrt(IN), (IN, HID)), rng.normal(0, 0.1, HID),
                      rng.normal(0, scale / np.sqrt(HID), (HID, HID)), rng.normal(0, 0.1, HID),
                      rng.normal(0, 1 / np.sqrt(HID), HID), 0.05)

    def blob(self) -> bytes:
        """Device parameter blob: W1 bf16, W2 bf16, b1, b2, w3 f32, b3 f32, padding."""
        parts = [bf16_bits(self.W1).tobytes(), bf16_bits(self.W2).tobytes(),
                 self.b1.astype(np.float32).tobytes(), self.b2.astype(np.float32).tobytes(),
                 self.w3.astype(np.float32).tobytes(), np.array([self.b3, 0, 0, 0], np.float32).tobytes()]
        return b"".join(parts)


def forward(p: Params, x, round_h1=True):
    """Returns (y, cache) for rows x [n, 32] (bf16 values).  round_h1=False
    gives the smooth network used for finite-difference checks."""
    x = bf16_round(x).astype(np.float64)
    z1 = x @ p.W1 + p.b1
    h1 = np.maximum(z1, 0.0)
    if round_h1:
        h1 = bf16_round(h1).astype(np.float64)
    z2 = h1 @ p.W2 + p.b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ p.w3 + p.b3
    return y, (x, z1, h1, z2, h2)


def logistic_loss(y, label, weight):
    """Weighted logistic loss sum_k weight_k * softplus(-(2 label_k - 1) y_k) and dL/dy."""
    s = 2.0 * np.asarray(label, np.float64) - 1.0
    m = -s * y
    loss = np.sum(weight * (np.maximum(m, 0) + np.log1p(np.exp(-np.abs(m)))))
    sig = 1.0 / (1.0 + np.exp(-y))
    dy = weight * (sig - label)
    return loss, dy


def backward(p: Params, cache, dy, bf16_operands=False):
    """Gradients of sum_k dy_k * y_k with respect to every parameter.  The
    bf16 rounding of h1 is treated as identity (straight-through), ReLU'(0) = 0.
    bf16_operands=True rounds dz2 and dz1 to bf16 where they enter the matrix
    products (as the tensor-core path does); the bias sums stay unrounded."""
    x, z1, h1, z2, h2 = cache
    rnd = (lambda a: bf16_round(a).astype(np.float64)) if bf16_operands else (lambda a: a)
    g = {}
    g["w3"] = h2.T @ dy
    g["b3"] = float(np.sum(dy))
    dh2 = np.outer(dy, p.w3)
    dz2 = dh2 * (z2 > 0)
    g["W2"] = h1.T @ rnd(dz2)
    g["b2"] = dz2.sum(axis=0)
    dh1 = rnd(dz2) @ p.W2.T
    dz1 = dh1 * (z1 > 0)
    g["W1"] = x.T @ rnd(dz1)
    g["b1"] = dz1.sum(axis=0)
    g["_abs"] = {"W2": np.abs(h1).T @ np.abs(dz2), "W1": np.abs(x).T @ np.abs(dz1),
                 "b2": np.abs(dz2).sum(axis=0), "b1": np.abs(dz1).sum(axis=0),
                 "w3": np.abs(h2).T @ np.abs(dy), "b3": float(np.abs(dy).sum())}
    return g


PARAM_ORDER = [("W1", (IN, HID)), ("W2", (HID, HID)), ("b1", (HID,)), ("b2", (HID,)), ("w3", (HID,)), ("b3", ())]
NUM_PARAMS = IN * HID + HID * HID + 3 * HID + 1


def split_vector(vec):
    """Parameter-order float vector (the device gradient layout) -> dict."""
    out, o = {}, 0
    for name, shape in PARAM_ORDER:
        k = int(np.prod(shape)) if shape else 1
        out[name] = vec[o:o + k].reshape(shape) if shape else float(vec[o])
        o += k
    return out


class Adam:
    """Adam (Kingma & Ba, "Adam: A Method for Stochastic Optimization", ICLR 2015,
    Algorithm 1) over a flat float64 parameter vector, written from its
    definition: m <- b1 m + (1 - b1) g;  v <- b2 v + (1 - b2) g^2;
    m_hat = m / (1 - b1^t);  v_hat = v / (1 - b2^t);
    theta <- theta - lr m_hat / (sqrt(v_hat) + eps), with t counted from 1."""

    def __init__(self, theta, beta1=0.9, beta2=0.999, eps=1e-8):
        self.theta = np.array(theta, dtype=np.float64)
        self.m = np.zeros_like(self.theta)
        self.v = np.zeros_like(self.theta)
        self.beta1, self.beta2, self.eps = float(beta1), float(beta2), float(eps)
        self.t = 0

    def step(self, grad, lr):
        g = np.asarray(grad, dtype=np.float64)
        self.t += 1
        self.m = self.beta1 * self.m + (1.0 - self.beta1) * g
        self.v = self.beta2 * self.v + (1.0 - self.beta2) * g * g
        m_hat = self.m / (1.0 - self.beta1 ** self.t)
        v_hat = self.v / (1.0 - self.beta2 ** self.t)
        self.theta = self.theta - lr * m_hat / (np.sqrt(v_hat) + self.eps)
        return self.theta
