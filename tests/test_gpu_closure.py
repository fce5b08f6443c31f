"""The learned warm start inside trt_step: trained on snapshots the method generates, it
changes where each step's iteration starts but not where it ends."""
import numpy as np
import pytest

from paper_2011_05427_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_05427_gb300 import build, closure, mlp, trt
    build.build()
    return torch, closure, mlp, trt


@pytest.fixture(scope="module")
def trained(env):
    torch, closure, mlp, trt = env
    slabs = [W.scaled(W.fc_small(), n, 8, 64, levels=[64, 16, 4, 1], name=f"t{n}")
             for n in (40, 90)]
    for c in slabs:
        c.dt, c.cycle, c.l_max = 1e-3, "V", 4
    X, Y = closure.collect(slabs, 10, 2048, seed=3)
    net, hist = closure.train(X, Y, iters=400, batch=2048, lr=2e-3)
    return net, hist


def test_training_on_method_snapshots(trained, env):
    net, hist = trained
    assert hist[-1][1] < 0.5 * hist[0][1], hist
    assert env[2].MLP.status() == 0


def test_warm_start_keeps_the_converged_answer(trained, env):
    """Warm-started steps converge to the plain method's state within the iteration
    tolerance's reach (eps = 1e-8 on both); the counters show what the warm start gains or
    loses (printed)."""
    torch, closure, mlp, trt = env
    net, _ = trained
    cfg = W.scaled(W.fc_small(), 60, 8, 64, levels=[64, 16, 4, 1])
    cfg.dt, cfg.cycle, cfg.l_max = 1e-3, "V", 4
    r = closure.compare(cfg, net, 8)
    a, b = r["plain"], r["closure"]
    dT = np.max(np.abs(a["state"]["T"] - b["state"]["T"]) / a["state"]["T"])
    E = a["state"]["Eg"].sum(0)
    dE = np.max(np.abs(a["state"]["Eg"] - b["state"]["Eg"]) / E[None, :])
    print(f"plain n_ti {a['n_ti']} n_c {a['n_c']}; closure n_ti {b['n_ti']} n_c {b['n_c']}; "
          f"dT {dT:.2e} dE {dE:.2e}")
    assert dT < 1e-6 and dE < 1e-6
    assert b["n_ti"] >= 8   # at least one sweep per step still closes the iteration


def test_removing_the_closure_restores_the_plain_path(trained, env):
    torch, closure, mlp, trt = env
    net, _ = trained
    cfg = W.scaled(W.fc_small(), 30, 4, 64, levels=[64, 16, 4, 1])
    a = trt.Solver.from_slab(cfg)
    b = trt.Solver.from_slab(cfg)
    b.set_closure(net)
    b.set_closure(None)
    for _ in range(3):
        sa = a.step(cfg.dt, "V", 4, 1e-8)
        sb = b.step(cfg.dt, "V", 4, 1e-8)
        assert (sa["n_ti"], sa["n_c"]) == (sb["n_ti"], sb["n_c"])
    assert np.array_equal(a.moments()["T"], b.moments()["T"])
