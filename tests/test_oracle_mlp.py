"""Pins of the FP64 surrogate-MLP oracle (CPU)."""
import math

import numpy as np

from oracle import mlp


def test_gelu_values():
    """GELU(z) = z Phi(z): Phi(0) = 1/2, Phi(1) = 0.841344746068543, Phi(-1) = 1 - Phi(1)."""
    z = np.array([0.0, 1.0, -1.0, 2.0])
    np.testing.assert_allclose(mlp.gelu(z), [0.0, 0.841344746068543, -0.158655253931457, 2 * 0.977249868051821],
                               rtol=1e-13, atol=1e-15)
    # derivative: Phi(z) + z phi(z); at 0 it is 1/2, at 1 it is Phi(1) + phi(1)
    np.testing.assert_allclose(mlp.gelu_grad(np.array([0.0, 1.0])),
                               [0.5, 0.841344746068543 + math.exp(-0.5) / math.sqrt(2 * math.pi)], rtol=1e-13)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    n_in, h, B = 12, 6, 5
    p = rng.normal(0, 0.5, mlp.n_params(n_in, h))
    X = rng.normal(0, 1, (B, n_in)); t = rng.normal(0, 1, B)
    _, g = mlp.loss_and_grad(p, X, t, n_in, h)
    eps = 1e-6
    fd = np.empty_like(p)
    for i in range(p.size):
        q = p.copy(); q[i] += eps
        lp, _ = mlp.loss_and_grad(q, X, t, n_in, h)
        q[i] -= 2 * eps
        lm, _ = mlp.loss_and_grad(q, X, t, n_in, h)
        fd[i] = (lp - lm) / (2 * eps)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-9)


def test_zero_hidden_weights_give_bias_output():
    """With W2 = 0 and b2 = 0 the hidden layer is GELU(0) = 0, so y = b3 for every input."""
    n_in, h = 8, 4
    p = np.zeros(mlp.n_params(n_in, h)); p[-1] = 0.75
    p[:h * n_in] = 1.0
    y, _ = mlp.forward(p, np.ones((3, n_in)), n_in, h)
    np.testing.assert_allclose(y, 0.75)


def test_adam_first_step_is_sign_step():
    """At t = 1 the bias-corrected moments are g and g^2, so the step is
    lr g / (|g| + eps), i.e. lr sign(g) up to eps."""
    g = np.array([3.0, -0.5, 1e-3, 0.0])
    p, m, v = mlp.adam(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.01, eps=1e-8)
    np.testing.assert_allclose(p, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g); np.testing.assert_allclose(v, 0.001 * g * g)


def test_one_hot_layout():
    oh = mlp.one_hot(np.array([[0, 3, 1]]))
    assert oh.shape == (1, 12)
    np.testing.assert_array_equal(oh[0], [1, 0, 0, 0, 0, 0, 0, 1, 0, 1, 0, 0])


def _torch_mlp(p, n_in, h):
    """The same network built from PyTorch's own FP64 layers (nn.Linear,
    exact-erf nn.GELU), with the flat parameter vector copied in."""
    import torch
    W1, b1, W2, b2, w3, b3 = mlp.unpack(p, n_in, h)
    net = torch.nn.Sequential(torch.nn.Linear(n_in, h), torch.nn.GELU(approximate="none"),
                              torch.nn.Linear(h, h), torch.nn.GELU(approximate="none"),
                              torch.nn.Linear(h, 1)).double()
    with torch.no_grad():
        for layer, (W, b) in zip((net[0], net[2], net[4]), ((W1, b1), (W2, b2), (w3[None, :], [b3]))):
            layer.weight.copy_(torch.tensor(np.asarray(W)))
            layer.bias.copy_(torch.tensor(np.asarray(b, np.float64)))
    return net


def _torch_flat(net, attr):
    return np.concatenate([getattr(t, attr).detach().numpy().ravel()
                           for t in (net[0].weight, net[0].bias, net[2].weight, net[2].bias,
                                     net[4].weight, net[4].bias)])


def test_forward_and_gradient_match_pytorch_fp64_layers():
    """A library definition of the same model: prediction, loss and the
    gradient of 0.5 mean (y - t)^2 from torch.autograd, in FP64.  A transposed
    weight, a dropped bias or a wrong activation fails here even when the
    oracle's own finite differences agree with it."""
    import torch
    rng = np.random.default_rng(4)
    n_in, h, B = 24, 10, 7
    p = rng.normal(0, 0.4, mlp.n_params(n_in, h))
    X = rng.normal(0, 1, (B, n_in)); t = rng.normal(0, 1, B)
    net = _torch_mlp(p, n_in, h)
    y_t = net(torch.tensor(X))[:, 0]
    loss_t = 0.5 * torch.mean((y_t - torch.tensor(t)) ** 2)
    loss_t.backward()
    y, _ = mlp.forward(p, X, n_in, h)
    loss, g = mlp.loss_and_grad(p, X, t, n_in, h)
    np.testing.assert_allclose(y, y_t.detach().numpy(), rtol=1e-13, atol=1e-14)
    assert abs(loss - loss_t.item()) <= 1e-13 * loss
    np.testing.assert_allclose(g, _torch_flat(net, "grad"), rtol=1e-11, atol=1e-14)


def test_adam_steps_match_pytorch_adam():
    """Five bias-corrected Adam steps against torch.optim.Adam (FP64) with the
    same hyper-parameters and gradients."""
    import torch
    rng = np.random.default_rng(9)
    p0 = rng.normal(0, 1, 40)
    grads = [rng.normal(0, 1, 40) * 10 ** rng.uniform(-3, 1, 40) for _ in range(5)]
    w = torch.tensor(p0.copy(), requires_grad=True)
    opt = torch.optim.Adam([w], lr=2e-3, betas=(0.8, 0.99), eps=1e-7)
    p, m, v = p0.copy(), np.zeros(40), np.zeros(40)
    for it, g in enumerate(grads, start=1):
        w.grad = torch.tensor(g)
        opt.step()
        p, m, v = mlp.adam(p, g, m, v, it, lr=2e-3, beta1=0.8, beta2=0.99, eps=1e-7)
        np.testing.assert_allclose(p, w.detach().numpy(), rtol=1e-13, atol=1e-15)
