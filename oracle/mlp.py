"""Oracle of the learned closure's network: plain numpy FP64 forward and backward passes.

THIS IS TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's CPU
baseline may import it; it shares nothing with the CUDA library.

The network (a learned warm start of the QD factors; the paper has no learned component):
    h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), h3 = relu(W3 h2 + b3),
    y = sigmoid(w4 . h3 + b4),  loss = (1/R) sum_r (y_r - t_r)^2.
Parameters use the flat layout of include/trt_mlp.h (W row-major [out][in]).

Two modes:
  exact  -- everything in FP64: the definition, pinned by finite differences;
  bf16   -- the same arithmetic, with values rounded to BF16 (round to nearest even) at the
            points where the tensor-core path stores them in BF16: the BF16 copies of W2,
            W3; the activations h1, h2 (and h3 where it multiplies dz in the w4 gradient);
            the layer gradients d3, d2 before they enter a product.
"""
import numpy as np

H = 256
OFF = dict(W1=0, b1=768, W2=1024, b2=66560, W3=66816, b3=132352, w4=132608, b4=132864)
NPARAM = 132868


def to_bf16(a):
    """Round to BF16 (the upper 16 bits of an IEEE binary32), ties to even, returned as
    float64.  Finite inputs only."""
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float64).astype(np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(p, hidden=H):
    """Split a flat parameter vector (hidden = 256: the trt_mlp.h layout; other sizes use
    the same order, packed without padding)."""
    p = np.asarray(p, dtype=np.float64)
    if hidden == H:
        o = OFF
    else:
        o, k = {}, 0
        for name, n in (("W1", 3 * hidden), ("b1", hidden), ("W2", hidden * hidden),
                        ("b2", hidden), ("W3", hidden * hidden), ("b3", hidden),
                        ("w4", hidden), ("b4", 1)):
            o[name] = k
            k += n
    return dict(W1=p[o["W1"]:o["W1"] + 3 * hidden].reshape(hidden, 3),
                b1=p[o["b1"]:o["b1"] + hidden],
                W2=p[o["W2"]:o["W2"] + hidden * hidden].reshape(hidden, hidden),
                b2=p[o["b2"]:o["b2"] + hidden],
                W3=p[o["W3"]:o["W3"] + hidden * hidden].reshape(hidden, hidden),
                b3=p[o["b3"]:o["b3"] + hidden],
                w4=p[o["w4"]:o["w4"] + hidden], b4=p[o["b4"]])


def nparam(hidden=H):
    return NPARAM if hidden == H else 3 * hidden + 2 * hidden * hidden + 4 * hidden + 1


def init_params(seed, hidden=H):
    """He-uniform weights, zero biases, a small last layer (f starts near 1/2)."""
    r = np.random.default_rng(seed)
    p = np.zeros(nparam(hidden))
    q = unpack(p, hidden)
    out = {}
    out["W1"] = r.uniform(-1, 1, (hidden, 3)) * np.sqrt(6.0 / 3)
    out["W2"] = r.uniform(-1, 1, (hidden, hidden)) * np.sqrt(6.0 / hidden)
    out["W3"] = r.uniform(-1, 1, (hidden, hidden)) * np.sqrt(6.0 / hidden)
    out["w4"] = r.uniform(-1, 1, hidden) * np.sqrt(1.0 / hidden)
    return pack({**{k: np.zeros_like(v) for k, v in q.items() if k != "b4"}, "b4": 0.0, **out},
                hidden)


def pack(d, hidden=H):
    p = np.zeros(nparam(hidden))
    if hidden == H:
        o = OFF
    else:
        o, k = {}, 0
        for name, n in (("W1", 3 * hidden), ("b1", hidden), ("W2", hidden * hidden),
                        ("b2", hidden), ("W3", hidden * hidden), ("b3", hidden),
                        ("w4", hidden), ("b4", 1)):
            o[name] = k
            k += n
    for name, v in d.items():
        v = np.atleast_1d(np.asarray(v, dtype=np.float64)).ravel()
        p[o[name]:o[name] + v.size] = v
    return p


def forward(p, x, mode="exact", hidden=H):
    """Returns y and the intermediates of the forward pass."""
    q = unpack(p, hidden)
    rb = to_bf16 if mode == "bf16" else (lambda a: np.asarray(a, dtype=np.float64))
    x = np.asarray(x, dtype=np.float64)
    a1 = x @ q["W1"].T + q["b1"]
    h1 = rb(np.maximum(a1, 0.0))
    a2 = h1 @ rb(q["W2"]).T + q["b2"]
    h2 = rb(np.maximum(a2, 0.0))
    a3 = h2 @ rb(q["W3"]).T + q["b3"]
    h3 = np.maximum(a3, 0.0)
    z = h3 @ q["w4"] + q["b4"]
    y = 1.0 / (1.0 + np.exp(-z))
    return y, dict(a1=a1, h1=h1, a2=a2, h2=h2, a3=a3, h3=h3, z=z)


def loss(p, x, t, mode="exact", hidden=H):
    y, _ = forward(p, x, mode, hidden)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def grad(p, x, t, mode="exact", hidden=H):
    """Gradient of loss() by the chain rule through the layers above (backward pass)."""
    q = unpack(p, hidden)
    rb = to_bf16 if mode == "bf16" else (lambda a: np.asarray(a, dtype=np.float64))
    x = np.asarray(x, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    R = x.shape[0]
    y, c = forward(p, x, mode, hidden)
    dz = (2.0 / R) * (y - t) * y * (1.0 - y)               # dL/dz
    d3 = rb(dz[:, None] * q["w4"][None, :] * (c["a3"] > 0))  # dL/da3
    g = {}
    g["w4"] = rb(c["h3"]).T @ dz
    g["b4"] = dz.sum()
    g["W3"] = d3.T @ c["h2"]
    g["b3"] = d3.sum(0)
    d2 = rb((d3 @ rb(q["W3"])) * (c["a2"] > 0))             # dL/da2
    g["W2"] = d2.T @ c["h1"]
    g["b2"] = d2.sum(0)
    d1 = (d2 @ rb(q["W2"])) * (c["a1"] > 0)                 # dL/da1
    g["W1"] = d1.T @ x
    g["b1"] = d1.sum(0)
    return pack(g, hidden), float(np.mean((y - t) ** 2))


def adam(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One bias-corrected Adam step (Kingma & Ba, Algorithm 1); returns new p, m, v."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def features(T, sigE, Eg):
    """Closure features per (group, cell) row, rows g-major: T [nx], sigE, Eg [G][nx]."""
    T = np.asarray(T, dtype=np.float64)
    sigE = np.asarray(sigE, dtype=np.float64)
    Eg = np.asarray(Eg, dtype=np.float64)
    E = Eg.sum(0)
    G, nx = sigE.shape
    x = np.empty((G, nx, 3))
    x[..., 0] = (np.log(np.maximum(T, 1e-30)) + 3.5) * 0.5
    x[..., 1] = (np.log(np.maximum(sigE, 1e-300)) - 10.0) * 0.1
    x[..., 2] = (np.log(np.maximum(Eg, 1e-300) / np.maximum(E, 1e-300)[None, :]) + 10.0) * 0.1
    return x.reshape(G * nx, 3)
