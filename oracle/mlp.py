"""FP64 reference of the capacity predictor's network -- TEST INFRASTRUCTURE ONLY.

The predictor maps a HyperLogLog sketch of a read set (1024 registers, each
divided by 64) to ln(distinct vertices) with a fully connected network
1024 -> 64 -> 64 -> 1, ReLU after the two hidden layers, trained on the mean
of (y - t)^2 / 2 with Adam (Kingma & Ba, "Adam: a method for stochastic
optimization", ICLR 2015, Algorithm 1, with its bias corrections).

The parameter vector is laid out W1[64][1024] | b1[64] | W2[64][64] | b2[64]
| w3[64] | b3, each weight matrix indexed [output][input].

Everything is plain numpy in float64: the forward pass is the definition, the
gradients are the chain rule written out layer by layer, and the Adam step is
the published update.  ``tests/test_oracle.py`` pins the gradients against
central finite differences and the forward pass and Adam step against closed
forms, so none of the three is checked only against itself.
"""

from __future__ import annotations

import numpy as np

IN, HID = 1024, 64
N_PARAMS = HID * IN + HID + HID * HID + HID + HID + 1


def unpack(p: np.ndarray) -> dict:
    """Views of the parameter vector's blocks (W1, b1, W2, b2, w3, b3)."""
    p = np.asarray(p, dtype=np.float64)
    if p.shape != (N_PARAMS,):
        raise ValueError(f"expected {N_PARAMS} parameters")
    o = 0
    out = {}
    for name, shape in (("W1", (HID, IN)), ("b1", (HID,)), ("W2", (HID, HID)), ("b2", (HID,)),
                        ("w3", (HID,)), ("b3", ())):
        n = int(np.prod(shape)) if shape else 1
        out[name] = p[o:o + n].reshape(shape) if shape else p[o]
        o += n
    return out


def pack(blocks: dict) -> np.ndarray:
    """Inverse of :func:`unpack`."""
    return np.concatenate([np.ravel(np.asarray(blocks[n], dtype=np.float64))
                           for n in ("W1", "b1", "W2", "b2", "w3", "b3")])


def forward(p: np.ndarray, x: np.ndarray) -> tuple[np.ndarray, dict]:
    """y[b] = w3 . relu(W2 relu(W1 x[b] + b1) + b2) + b3, with the hidden
    pre-activations and activations for the backward pass."""
    q = unpack(p)
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ q["W1"].T + q["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ q["W2"].T + q["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ q["w3"] + q["b3"]
    return y, {"x": x, "z1": z1, "h1": h1, "z2": z2, "h2": h2}


def loss(p: np.ndarray, x: np.ndarray, t: np.ndarray) -> float:
    """Mean over the batch of (y - t)^2 / 2."""
    y, _ = forward(p, x)
    d = y - np.asarray(t, dtype=np.float64)
    return float(0.5 * np.mean(d * d))


def loss_and_grads(p: np.ndarray, x: np.ndarray, t: np.ndarray) -> tuple[float, np.ndarray]:
    """The loss and its gradient with respect to every parameter (chain rule;
    the ReLU's derivative is taken as 0 at 0)."""
    q = unpack(p)
    y, c = forward(p, x)
    B = y.shape[0]
    d = y - np.asarray(t, dtype=np.float64)
    dy = d / B
    g = {"w3": c["h2"].T @ dy, "b3": dy.sum()}
    dz2 = np.outer(dy, q["w3"]) * (c["z2"] > 0)
    g["W2"] = dz2.T @ c["h1"]
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ q["W2"]) * (c["z1"] > 0)
    g["W1"] = dz1.T @ c["x"]
    g["b1"] = dz1.sum(axis=0)
    return float(0.5 * np.mean(d * d)), pack(g)


def adam_step(p, g, m, v, step: int, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update (step >= 1): returns new (p, m, v)."""
    m = beta1 * np.asarray(m, dtype=np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, dtype=np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return np.asarray(p, dtype=np.float64) - lr * mhat / (np.sqrt(vhat) + eps), m, v


def abs_forward(p: np.ndarray, x: np.ndarray) -> np.ndarray:
    """The same network with every weight, bias and input replaced by its
    absolute value and no ReLU: the magnitude that bounds the rounding error
    of a float32 evaluation (each dot product of n terms is off by at most
    about n * 2^-24 times the sum of its terms' magnitudes)."""
    q = {n: np.abs(a) for n, a in unpack(p).items()}
    a1 = np.abs(x) @ q["W1"].T + q["b1"]
    a2 = a1 @ q["W2"].T + q["b2"]
    return a2 @ q["w3"] + q["b3"]
