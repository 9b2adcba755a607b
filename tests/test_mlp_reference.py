"""Pins for the float64 MLP reference (oracle/mlp.py) on the CPU.

The reference's analytic gradient must match central finite differences of
its own loss on a tiny network, and its features must be the definition
x = [a xor b, a and b] (checked bit by bit against Python integers).
"""
import numpy as np

from oracle import mlp


def test_features_definition():
    rng = np.random.default_rng(0)
    vec = rng.integers(0, 2 ** 32, size=(5, 2), dtype=np.uint64).astype(np.uint32)
    x = mlp.features(vec, np.array([0, 3]), np.array([1, 4]))
    for row, (i, j) in enumerate([(0, 1), (3, 4)]):
        a = int(vec[i, 0]) | (int(vec[i, 1]) << 32)
        b = int(vec[j, 0]) | (int(vec[j, 1]) << 32)
        for f in range(64):
            assert x[row, f] == ((a ^ b) >> f) & 1
            assert x[row, 64 + f] == ((a & b) >> f) & 1


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    F, H = 64, 6            # one 32-bit word per vector
    n = F * H + H + H * H + H + H + 1
    params = rng.normal(scale=0.3, size=n)
    vec = rng.integers(0, 2 ** 32, size=(7, 1), dtype=np.uint64).astype(np.uint32)
    pa, pb = np.array([0, 1, 2, 3, 4]), np.array([5, 6, 0, 1, 2])
    y = np.array([1, 0, 1, 0, 0], np.float64)
    w = np.array([1.0, 2.0, 0.5, 1.0, 3.0])
    loss, grad = mlp.loss_and_grad(params, F, H, vec, pa, pb, y, w)
    eps = 1e-6
    for i in rng.choice(n, 60, replace=False):
        p1, p2 = params.copy(), params.copy()
        p1[i] += eps
        p2[i] -= eps
        num = (mlp.loss_and_grad(p1, F, H, vec, pa, pb, y, w)[0] - mlp.loss_and_grad(p2, F, H, vec, pa, pb, y, w)[0]) / (2 * eps)
        assert abs(num - grad[i]) <= 1e-6 * max(1.0, abs(num)), i
    # the loss is the weighted binary cross-entropy of the forward logits
    z = mlp.forward(params, F, H, vec, pa, pb)
    want = np.sum(w * (np.log1p(np.exp(z)) - y * z))
    assert abs(loss - want) < 1e-9
