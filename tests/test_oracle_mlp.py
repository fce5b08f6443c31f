"""Pins of the MLP oracle (oracle/mlp.py) against things other than itself: the BF16
format's definition and a library conversion, finite differences of the loss, the Adam
update's closed form on its first step, and the features' definition at known states."""
import numpy as np
import pytest

from oracle import mlp as M


def test_bf16_rounding_definition():
    # spacing of BF16 at 1 is 2^-7; halfway cases go to the even significand
    cases = [(1.0, 1.0), (1 + 2 ** -8, 1.0), (1 + 3 * 2 ** -8, 1 + 2 ** -6),
             (1 + 2 ** -8 + 2 ** -20, 1 + 2 ** -7), (-(1 + 2 ** -7), -(1 + 2 ** -7)),
             (3.0, 3.0), (0.0, 0.0), (2.0 ** -130, 2.0 ** -130)]
    for a, b in cases:
        assert M.to_bf16(np.array([a]))[0] == b, (a, b)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    r = np.random.default_rng(3)
    a = (r.standard_normal(20000) * np.exp(r.uniform(-20, 20, 20000))).astype(np.float32)
    ref = torch.from_numpy(a).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.to_bf16(a), ref)


def _problem(hidden, R, seed):
    r = np.random.default_rng(seed)
    p = M.init_params(seed, hidden)
    p = p + M.pack({"b1": r.normal(0, 0.1, hidden), "b2": r.normal(0, 0.1, hidden),
                    "b3": r.normal(0, 0.1, hidden), "b4": 0.3}, hidden) * 1.0
    x = r.normal(0, 1, (R, 3))
    t = r.uniform(0.3, 1.0, R)
    return p, x, t


@pytest.mark.parametrize("hidden", [4, 8])
def test_exact_gradient_against_finite_differences(hidden):
    p, x, t = _problem(hidden, 16, 7 + hidden)
    g, L = M.grad(p, x, t, "exact", hidden)
    assert L == pytest.approx(M.loss(p, x, t, "exact", hidden), rel=1e-14)
    h = 1e-6
    for k in range(p.size):
        e = np.zeros_like(p)
        e[k] = h
        fd = (M.loss(p + e, x, t, "exact", hidden) - M.loss(p - e, x, t, "exact", hidden)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1e-3, np.abs(g).max()), (k, fd, g[k])


def test_exact_gradient_full_width_sampled():
    p, x, t = _problem(256, 24, 11)
    g, _ = M.grad(p, x, t)
    r = np.random.default_rng(12)
    blocks = [(M.OFF["W1"], 768), (M.OFF["b1"], 256), (M.OFF["W2"], 65536), (M.OFF["b2"], 256),
              (M.OFF["W3"], 65536), (M.OFF["b3"], 256), (M.OFF["w4"], 256), (M.OFF["b4"], 1)]
    h = 1e-6
    for off, n in blocks:
        for k in off + r.choice(n, min(n, 6), replace=False):
            e = np.zeros_like(p)
            e[k] = h
            fd = (M.loss(p + e, x, t) - M.loss(p - e, x, t)) / (2 * h)
            assert abs(fd - g[k]) <= 1e-6 * max(1e-4, abs(g).max()), (k, fd, g[k])


def test_bf16_mode_is_close_to_exact():
    p, x, t = _problem(256, 64, 13)
    ge, _ = M.grad(p, x, t, "exact")
    gb, _ = M.grad(p, x, t, "bf16")
    assert np.linalg.norm(gb - ge) < 3e-2 * np.linalg.norm(ge)
    ye, _ = M.forward(p, x, "exact")
    yb, _ = M.forward(p, x, "bf16")
    assert np.max(np.abs(yb - ye)) < 1e-2


def test_adam_first_step_closed_form():
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    p1, m, v = M.adam(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, 0.01)
    # first bias-corrected step: m_hat = g, v_hat = g^2, update = lr g / (|g| + eps)
    assert np.allclose(p1, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)


def test_features_definition():
    T = np.array([np.exp(-3.5), 1.0])
    sig = np.array([[np.exp(10.0), 1.0], [np.exp(20.0), np.exp(-10.0)]])
    Eg = np.array([[1.0, 3.0], [1.0, 1.0]])
    x = M.features(T, sig, Eg).reshape(2, 2, 3)
    assert np.allclose(x[0, 0], [0.0, 0.0, (np.log(0.5) + 10) * 0.1])
    assert np.allclose(x[1, 1], [1.75, -2.0, (np.log(0.25) + 10) * 0.1])
