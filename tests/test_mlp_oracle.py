"""Pins of the fp64 reference network: gradient by finite differences, forward by per-neuron loops."""
import numpy as np

from oracle import mlp as M


def _params(rng):
    return rng.normal(0, 0.3, M.N_PARAMS)


def test_forward_matches_per_neuron_loops():
    rng = np.random.default_rng(1)
    flat = _params(rng)
    X = rng.normal(0, 1, (5, M.IN))
    y, _ = M.forward(flat, X)
    p = M.unpack(flat)
    for s in range(5):
        h1 = [max(0.0, p["b1"][i] + sum(p["W1"][i][j] * X[s][j] for j in range(M.IN))) for i in range(M.HID)]
        h2 = [max(0.0, p["b2"][i] + sum(p["W2"][i][j] * h1[j] for j in range(M.HID))) for i in range(M.HID)]
        want = p["b3"][0] + sum(p["W3"][i] * h2[i] for i in range(M.HID))
        assert abs(y[s] - want) < 1e-12 * max(1.0, abs(want))


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    flat = _params(rng)
    X = rng.normal(0, 1, (7, M.IN))
    t = rng.normal(0, 1, 7)
    scale = 1.0 / 7
    _, g = M.loss_and_grad(flat, X, t, scale)
    h = 1e-6
    for idx in list(rng.choice(M.N_PARAMS, 60, replace=False)) + [0, 1023, 1024, 1087, 1088, 5183, 5184, 5248, 5312]:
        e = np.zeros(M.N_PARAMS)
        e[idx] = h
        lp, _ = M.loss_and_grad(flat + e, X, t, scale)
        lm, _ = M.loss_and_grad(flat - e, X, t, scale)
        fd = scale * (lp - lm) / (2 * h)
        assert abs(fd - g[idx]) <= 1e-6 * max(1.0, abs(g[idx])), idx


def test_bf16_widening_is_exact():
    bits = np.array([0x3F80, 0xBF80, 0x4049, 0x0000, 0x7F7F], dtype=np.uint16)   # 1, -1, ~3.14, 0, max
    v = M.bf16_to_f64(bits)
    assert v[0] == 1.0 and v[1] == -1.0 and v[3] == 0.0
    assert abs(v[2] - 3.140625) < 1e-12 and v[4] > 3e38
