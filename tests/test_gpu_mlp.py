"""The learned closure's tensor-core kernels (trt_gemm_bf16, trt_mlp_*) against plain
numpy FP64 arithmetic and the MLP oracle, through the C ABI."""
import numpy as np
import pytest

from oracle import mlp as OM

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_05427_gb300 import build, mlp
    build.build()
    return torch, mlp


def bf16_dev(torch, a):
    return torch.as_tensor(np.asarray(a, np.float32)).to(torch.bfloat16).cuda()


@pytest.mark.parametrize("M,N,K", [(128, 256, 64), (300, 256, 256), (1000, 512, 256),
                                   (256, 256, 4096), (5, 256, 128)])
def test_gemm_plain(env, M, N, K):
    """FP32 accumulation of BF16 products: equal to the FP64 product of the BF16 inputs up
    to FP32 rounding of the K-term sum."""
    torch, mlp = env
    r = np.random.default_rng(M + N + K)
    A = OM.to_bf16(r.normal(0, 1, (M, K)))
    B = OM.to_bf16(r.normal(0, 1, (N, K)))
    c32, _, _ = mlp.gemm_bf16(bf16_dev(torch, A), bf16_dev(torch, B))
    ref = A @ B.T
    got = c32.cpu().numpy().astype(np.float64)
    scale = np.sqrt((A * A).sum(1))[:, None] * np.sqrt((B * B).sum(1))[None, :]
    assert np.max(np.abs(got - ref) / scale) < 1e-5


def test_gemm_epilogue(env):
    torch, mlp = env
    M, N, K = 260, 256, 192
    r = np.random.default_rng(5)
    A = OM.to_bf16(r.normal(0, 1, (M, K)))
    B = OM.to_bf16(r.normal(0, 1, (N, K)))
    bias = r.normal(0, 1, N).astype(np.float32)
    mask = OM.to_bf16(r.normal(0, 1, (M, N)))
    o32, o16, o16T = mlp.gemm_bf16(bf16_dev(torch, A), bf16_dev(torch, B),
                                   bias=torch.as_tensor(bias).cuda(), relu=True,
                                   mask=bf16_dev(torch, mask), out32=True, out16=True, out16T=True)
    ref = np.maximum(A @ B.T + bias, 0.0) * (mask > 0)
    got = o32.cpu().numpy()
    scale = np.sqrt((A * A).sum(1))[:, None] * np.sqrt((B * B).sum(1))[None, :] + np.abs(bias)
    assert np.max(np.abs(got - ref) / scale) < 1e-5
    g16 = o16.float().cpu().numpy()
    assert np.array_equal(g16, OM.to_bf16(got))
    assert np.array_equal(o16T.float().cpu().numpy(), g16.T)


def test_mlp_forward_vs_oracle(env):
    torch, mlp = env
    p = OM.init_params(21)
    r = np.random.default_rng(22)
    p = p + OM.pack({"b1": r.normal(0, 0.1, 256), "b2": r.normal(0, 0.1, 256),
                     "b3": r.normal(0, 0.1, 256), "b4": 0.2})
    p32 = p.astype(np.float32).astype(np.float64)
    x = r.normal(0, 1, (1000, 3)).astype(np.float32)
    net = mlp.MLP(p32)
    y = net.forward(x).cpu().numpy()
    ref, _ = OM.forward(p32, x.astype(np.float64), "bf16")
    assert np.max(np.abs(y - ref)) < 2e-3
    assert mlp.MLP.status() == 0


@pytest.mark.parametrize("rows", [1, 1000, 100000])
def test_mlp_fused_forward(env, rows):
    """The persistent fused kernel against the three-launch path (same arithmetic, same
    accumulation order) and the oracle; 1000 rows end in a partial 256-row tile, 100000
    rows give every CTA several tiles."""
    torch, mlp = env
    p = OM.init_params(61)
    r = np.random.default_rng(62)
    p = p + OM.pack({"b1": r.normal(0, 0.1, 256), "b2": r.normal(0, 0.1, 256),
                     "b3": r.normal(0, 0.1, 256), "b4": -0.3})
    p32 = p.astype(np.float32).astype(np.float64)
    x = r.normal(0, 1, (rows, 3)).astype(np.float32)
    net = mlp.MLP(p32)
    yf = net.forward_fused(x).cpu().numpy()
    y3 = net.forward(x).cpu().numpy()
    assert np.max(np.abs(yf - y3)) < 1e-6
    k = min(rows, 2000)
    ref, _ = OM.forward(p32, x[:k].astype(np.float64), "bf16")
    assert np.max(np.abs(yf[:k] - ref)) < 2e-3
    assert mlp.MLP.status() == 0


def test_mlp_gradient_vs_oracle(env):
    """Gradients of the tensor-core backward pass against the oracle's backward pass with
    BF16 rounding at the same points, element by element: every element within 5e-4 of its
    parameter block's largest gradient (measured up to 7.7e-5: FP32 accumulation order,
    and BF16 roundings of stored activations that flip with it), and the block norms
    within 2e-3."""
    torch, mlp = env
    r = np.random.default_rng(31)
    p = OM.init_params(30) + OM.pack({"b1": r.normal(0, 0.1, 256), "b2": r.normal(0, 0.1, 256),
                                      "b3": r.normal(0, 0.1, 256), "b4": 0.2})
    p32 = p.astype(np.float32).astype(np.float64)
    R = 512
    x = r.normal(0, 1, (R, 3)).astype(np.float32)
    t = r.uniform(0.3, 1.0, R).astype(np.float32)
    net = mlp.MLP(p32)
    g, L = net.grad(x, t)
    g = g.cpu().numpy().astype(np.float64)
    gr, Lr = OM.grad(p32, x.astype(np.float64), t.astype(np.float64), "bf16")
    assert L.item() == pytest.approx(Lr, rel=1e-3)
    for name, n in (("W1", 768), ("b1", 256), ("W2", 65536), ("b2", 256), ("W3", 65536),
                    ("b3", 256), ("w4", 256), ("b4", 1)):
        o = OM.OFF[name]
        a, b = g[o:o + n], gr[o:o + n]
        scale = np.abs(b).max() + 1e-30
        elem = np.abs(a - b) / scale
        print(f"{name}: max element error {elem.max():.2e}, 99th percentile "
              f"{np.quantile(elem, 0.99):.2e} of the block's largest gradient")
        assert elem.max() <= 5e-4, name
        assert np.linalg.norm(a - b) <= 2e-3 * np.linalg.norm(b) + 1e-12, name
    assert mlp.MLP.status() == 0


def test_adam_step_vs_oracle(env):
    torch, mlp = env
    r = np.random.default_rng(41)
    p = OM.init_params(40).astype(np.float32).astype(np.float64)
    R = 256
    x = r.normal(0, 1, (R, 3)).astype(np.float32)
    t = r.uniform(0.3, 1.0, R).astype(np.float32)
    net = mlp.MLP(p)
    g, _ = net.grad(x, t)
    g = g.cpu().numpy().astype(np.float64)
    net.adam_step(lr=1e-3)
    pr, _, _ = OM.adam(p, g, np.zeros_like(p), np.zeros_like(p), 1, 1e-3)
    got = net.params.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - pr)) < 1e-6
    # the BF16 copies follow the FP32 master weights
    w16 = net.w16.float().cpu().numpy()
    W2 = OM.unpack(got)["W2"]
    assert np.array_equal(w16[:65536].reshape(256, 256), OM.to_bf16(W2))
    assert np.array_equal(w16[2 * 65536:3 * 65536].reshape(256, 256), OM.to_bf16(W2).T)


def test_training_reduces_loss(env):
    """A few hundred Adam steps on a smooth target of the features lower the loss 10x."""
    torch, mlp = env
    r = np.random.default_rng(51)
    R = 2048
    x = r.uniform(-1.5, 1.5, (R, 3)).astype(np.float32)
    t = (0.35 + 0.5 / (1 + np.exp(-2 * x[:, 1] + x[:, 2])) + 0.1 * np.tanh(x[:, 0])).astype(np.float32)
    t = np.clip(t, 0.34, 0.99)
    net = mlp.MLP(OM.init_params(50))
    L0 = net.grad(x, t)[1].item()
    for _ in range(300):
        net.train_step(x, t, lr=1e-3)
    L1 = net.grad(x, t)[1].item()
    assert L1 < 0.1 * L0, (L0, L1)
    assert mlp.MLP.status() == 0
