"""FP64 reference of the learned temperature inversion T(rho, e) (test
infrastructure only; the CUDA path never imports it).

Network (2 -> 64 -> 64 -> 1, tanh hidden units), on normalised inputs:
    x0 = (log rho - c_rho) / s_rho,  x1 = (e - c_e) / s_e
    h1 = tanh(W1 x + b1),  h2 = tanh(W2 h1 + b2),  y = W3 . h2 + b3
    T_hat = c_T + s_T y
Parameters are one float array in the library's order:
    [c_rho, s_rho, c_e, s_e, c_T, s_T | W1 (64x2) | b1 (64) | W2 (64x64, [out][in]) | b2 (64) | W3 (64) | b3]
Loss: mean over the batch of (y - t)^2 / 2 with t = (T - c_T)/s_T.

bf16=True evaluates the same network at the precision of the library's
tensor-core products: the operands those products read (W2, h1, and in the
backward pass delta2) are rounded to bfloat16 (from their float32 value,
nearest, ties to even), everything else stays FP64.  This is the "FP32-cast
weights with BF16 inputs" reference of the gradient parity check; the
gradient is that of the rounded computation with the roundings held fixed.
"""
from __future__ import annotations

import numpy as np

H = 64
N_NORM = 6
SIZES = [("W1", (H, 2)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H,)), ("b3", (1,))]
N_PARAMS = N_NORM + sum(int(np.prod(s)) for _, s in SIZES)


def bf16(x) -> np.ndarray:
    """Round to bfloat16 (8-bit significand): the float32 value's upper 16
    bits after round-to-nearest, ties to even (IEEE rounding of the 23-bit
    fraction to 7 bits), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return (r & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(p: np.ndarray) -> dict:
    p = np.asarray(p, dtype=np.float64)
    out = {"norm": p[:N_NORM]}
    o = N_NORM
    for name, shape in SIZES:
        n = int(np.prod(shape))
        out[name] = p[o:o + n].reshape(shape)
        o += n
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d["norm"], dtype=np.float64)] +
                          [np.asarray(d[name], dtype=np.float64).ravel() for name, _ in SIZES])


def init_params(rho_range, e_range, T_range, seed: int = 0) -> np.ndarray:
    """Normalisation from the sample box; weights ~ U(-1/sqrt(fan_in), ...)."""
    rng = np.random.default_rng(seed)
    lr0, lr1 = np.log(rho_range[0]), np.log(rho_range[1])
    norm = [0.5 * (lr0 + lr1), 0.5 * (lr1 - lr0), 0.5 * (e_range[0] + e_range[1]),
            0.5 * (e_range[1] - e_range[0]), 0.5 * (T_range[0] + T_range[1]), 0.5 * (T_range[1] - T_range[0])]
    d = {"norm": np.array(norm)}
    for name, shape in SIZES:
        fan_in = shape[1] if len(shape) == 2 else (H if name == "W3" else 1)
        lim = 1.0 / np.sqrt(fan_in)
        d[name] = rng.uniform(-lim, lim, shape) if name[0] == "W" else np.zeros(shape)
    return pack(d)


def features(p: np.ndarray, rho, e):
    n = unpack(p)["norm"]
    return np.stack([(np.log(rho) - n[0]) / n[1], (np.asarray(e) - n[2]) / n[3]], axis=-1)


def forward(p: np.ndarray, rho, e, bf16_products: bool = False):
    """T_hat and the intermediate activations."""
    d = unpack(p)
    x = features(p, rho, e)
    h1 = np.tanh(x @ d["W1"].T + d["b1"])
    if bf16_products:
        h2 = np.tanh(bf16(h1) @ bf16(d["W2"]).T + d["b2"])
    else:
        h2 = np.tanh(h1 @ d["W2"].T + d["b2"])
    y = h2 @ d["W3"] + d["b3"][0]
    n = d["norm"]
    return n[4] + n[5] * y, (x, h1, h2, y)


def loss_and_grad(p: np.ndarray, rho, e, T, bf16_products: bool = False):
    """Mean squared error of the normalised output and its gradient with
    respect to the trainable parameters (normalisation entries get 0)."""
    d = unpack(p)
    n = d["norm"]
    _, (x, h1, h2, y) = forward(p, rho, e, bf16_products)
    # operands of the two products through W2 (forward h1 . W2^T; backward delta2 . W2, delta2^T . h1)
    rnd = bf16 if bf16_products else (lambda v: v)
    W2 = rnd(d["W2"])
    t = (np.asarray(T) - n[4]) / n[5]
    B = y.shape[0]
    r = y - t
    loss = 0.5 * np.mean(r * r)
    d3 = r / B                                  # dL/dy
    g = {"norm": np.zeros(N_NORM)}
    g["W3"] = h2.T @ d3
    g["b3"] = np.array([d3.sum()])
    d2 = np.outer(d3, d["W3"]) * (1.0 - h2 * h2)
    g["W2"] = rnd(d2).T @ rnd(h1)
    g["b2"] = d2.sum(axis=0)
    d1 = (rnd(d2) @ W2) * (1.0 - h1 * h1)
    g["W1"] = d1.T @ x
    g["b1"] = d1.sum(axis=0)
    return loss, pack(g)


def adam_train(p: np.ndarray, rho, e, T, epochs: int, batch: int, lr: float, seed: int = 0):
    """Plain Adam (beta1 0.9, beta2 0.999, eps 1e-8) on shuffled minibatches."""
    p = np.array(p, dtype=np.float64)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    rng = np.random.default_rng(seed)
    t = 0
    n = len(rho)
    for _ in range(epochs):
        order = rng.permutation(n)
        for s in range(0, n - batch + 1, batch):
            idx = order[s:s + batch]
            _, g = loss_and_grad(p, rho[idx], e[idx], T[idx])
            t += 1
            m = 0.9 * m + 0.1 * g
            v = 0.999 * v + 0.001 * g * g
            mh = m / (1 - 0.9 ** t)
            vh = v / (1 - 0.999 ** t)
            upd = lr * mh / (np.sqrt(vh) + 1e-8)
            upd[:N_NORM] = 0.0
            p -= upd
    return p
