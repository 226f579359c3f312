"""Pins of the surrogate-network oracle (CPU only): analytic gradients
against central finite differences in FP64, the forward pass against torch's
independent Linear/GELU implementation, the bfloat16 rounding against
torch's conversion, and Adam against torch.optim.Adam."""
import numpy as np
import pytest

from oracle import mlp


def data(B, seed):
    r = np.random.default_rng(seed)
    X = r.normal(0, 1, (B, 16))
    y = (r.random(B) < 0.6).astype(np.float64)
    t = r.random(B)
    mask = (1 - y)
    return X, y, t, mask


def test_param_count():
    assert mlp.N_PARAMS == 202242


def test_gradients_vs_finite_differences():
    """Without bf16 rounding the loss is smooth: central differences (step
    1e-6) agree with the analytic gradient to 1e-6 relative on sampled
    parameters of every tensor."""
    X, y, t, mask = data(32, 1)
    p = mlp.init_params(3)
    out, cache = mlp.forward(p, X, bf16_points=False)
    L, d = mlp.loss_and_dout(out, y, t, mask, 0.7)
    g = mlp.backward(p, cache, d, bf16_points=False)
    rng = np.random.default_rng(2)
    off = 0
    for s in mlp.param_shapes():
        n = int(np.prod(s))
        for j in rng.choice(n, min(4, n), replace=False):
            i = off + j
            h = 1e-6
            pp, pm = p.copy(), p.copy()
            pp[i] += h
            pm[i] -= h
            Lp = mlp.loss_and_dout(mlp.forward(pp, X, False)[0], y, t, mask, 0.7)[0]
            Lm = mlp.loss_and_dout(mlp.forward(pm, X, False)[0], y, t, mask, 0.7)[0]
            fd = (Lp - Lm) / (2 * h)
            assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-10), (s, j)
        off += n


def test_forward_and_backward_vs_torch():
    torch = pytest.importorskip("torch")
    X, y, t, mask = data(64, 4)
    p = mlp.init_params(5)
    ps = [torch.tensor(a, dtype=torch.float64, requires_grad=True) for a in mlp.unflatten(p)]
    h = torch.tensor(X)
    for l in range(4):
        h = torch.nn.functional.gelu(torch.nn.functional.linear(h, ps[2 * l], ps[2 * l + 1]))
    o = torch.nn.functional.linear(h, ps[8], ps[9])
    bce = torch.nn.functional.binary_cross_entropy_with_logits(o[:, 0], torch.tensor(y))
    m = torch.tensor(mask)
    L = bce + 0.7 * torch.sum(m * (o[:, 1] - torch.tensor(t)) ** 2) / max(float(mask.sum()), 1.0)
    L.backward()
    out, cache = mlp.forward(p, X, bf16_points=False)
    Lo, d = mlp.loss_and_dout(out, y, t, mask, 0.7)
    g = mlp.backward(p, cache, d, bf16_points=False)
    assert np.allclose(out, o.detach().numpy(), rtol=1e-12, atol=1e-14)
    assert Lo == pytest.approx(float(L), rel=1e-12)
    gt = np.concatenate([q.grad.numpy().reshape(-1) for q in ps])
    assert np.allclose(g, gt, rtol=1e-9, atol=1e-15)


def test_bf16_rounding_vs_torch():
    torch = pytest.importorskip("torch")
    v = np.random.default_rng(6).normal(0, 10, 100000).astype(np.float32)
    v[:4] = [0.0, -0.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8]  # ties round to even
    ref = torch.tensor(v).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(v), ref)


def test_adam_vs_torch():
    torch = pytest.importorskip("torch")
    r = np.random.default_rng(7)
    p0 = r.normal(0, 1, 50)
    w = torch.tensor(p0.copy(), requires_grad=True)
    opt = torch.optim.Adam([w], lr=1e-2)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for step in range(1, 6):
        g = r.normal(0, 1, 50)
        w.grad = torch.tensor(g)
        opt.step()
        p, m, v = mlp.adam(p, g, m, v, step, 1e-2)
    assert np.allclose(p, w.detach().numpy(), rtol=1e-12, atol=1e-14)
