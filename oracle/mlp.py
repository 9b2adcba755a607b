"""Float64 reference of the pair-ranking MLP -- TEST INFRASTRUCTURE.

The same network as libmk's kernels, written as plain numpy in float64 so
the GPU's FP32 forward pass and gradients can be checked against it: for a
pair (a, b) of truth vectors (bit arrays), x = [a xor b, a and b];
h1 = relu(x W1 + b1); h2 = relu(h1 W2 + b2); z = h2 . w3 + b3; the loss is
the weighted binary cross-entropy sum_i w_i (log(1 + e^z_i) - y_i z_i).
Parameters are one flat vector in the order W1[F][H], b1, W2[H][H], b2,
w3[H], b3.
"""
import numpy as np


def unpack(params, F, H):
    p = np.asarray(params, np.float64)
    i = 0
    W1 = p[i:i + F * H].reshape(F, H); i += F * H
    b1 = p[i:i + H]; i += H
    W2 = p[i:i + H * H].reshape(H, H); i += H * H
    b2 = p[i:i + H]; i += H
    w3 = p[i:i + H]; i += H
    b3 = p[i]
    return W1, b1, W2, b2, w3, b3


def features(vec_words, pa, pb):
    """x[i] = [a xor b, a and b] as 0/1 float64; vec_words: uint32 [nvec][words]."""
    bits = np.unpackbits(np.ascontiguousarray(vec_words).view(np.uint8), axis=1, bitorder="little")
    a, b = bits[pa], bits[pb]
    return np.concatenate([a ^ b, a & b], axis=1).astype(np.float64)


def forward(params, F, H, vec_words, pa, pb):
    W1, b1, W2, b2, w3, b3 = unpack(params, F, H)
    x = features(vec_words, pa, pb)
    h1 = np.maximum(x @ W1 + b1, 0.0)
    h2 = np.maximum(h1 @ W2 + b2, 0.0)
    return h2 @ w3 + b3


def loss_and_grad(params, F, H, vec_words, pa, pb, y, w=None):
    W1, b1, W2, b2, w3, b3 = unpack(params, F, H)
    w = np.ones(len(pa)) if w is None else np.asarray(w, np.float64)
    y = np.asarray(y, np.float64)
    x = features(vec_words, pa, pb)
    h1 = np.maximum(x @ W1 + b1, 0.0)
    h2 = np.maximum(h1 @ W2 + b2, 0.0)
    z = h2 @ w3 + b3
    loss = float(np.sum(w * (np.logaddexp(0.0, z) - y * z)))
    dz = w * (1.0 / (1.0 + np.exp(-z)) - y)
    gw3 = h2.T @ dz
    gb3 = dz.sum()
    dh2 = np.outer(dz, w3) * (h2 > 0)
    gW2 = h1.T @ dh2
    gb2 = dh2.sum(0)
    dh1 = (dh2 @ W2.T) * (h1 > 0)
    gW1 = x.T @ dh1
    gb1 = dh1.sum(0)
    grad = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gw3, [gb3]])
    return loss, grad
