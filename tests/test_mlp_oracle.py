"""Pins of the surrogate's MLP oracle against things other than itself:
finite differences of its loss, closed forms of GELU, a library bf16
conversion, a brute-force loop forward, and the zero-residual case."""
import math

import numpy as np
import pytest

from oracle.mlp_oracle import MLPOracle, bf16_round, gelu, gelu_grad


def net_and_data(seed=0, n_in=6, width=12, depth=3, n_out=5, n=9):
    o = MLPOracle(n_in, width, depth, n_out)
    rng = np.random.default_rng(seed)
    p = rng.normal(0.0, 0.4, o.param_count())
    X = rng.normal(size=(n, n_in))
    T = rng.normal(size=(n, n_out))
    w = rng.uniform(0.5, 2.0, n_out)
    return o, p, X, T, w


def test_gradient_matches_central_differences_fp64():
    o, p, X, T, w = net_and_data()
    loss, g = o.loss_grad(p, X, T, w, bf16=False)
    assert loss == pytest.approx(o.loss(p, X, T, w, bf16=False), rel=1e-15)
    rng = np.random.default_rng(3)
    idx = rng.choice(p.size, 60, replace=False)
    h = 1e-6
    for q in idx:
        e = np.zeros_like(p)
        e[q] = h
        fd = (o.loss(p + e, X, T, w, bf16=False) - o.loss(p - e, X, T, w, bf16=False)) / (2 * h)
        assert abs(fd - g[q]) <= 1e-7 * max(1.0, abs(g[q])), (q, fd, g[q])


def test_every_layer_gets_gradient_and_layout_is_layerwise():
    o, p, X, T, w = net_and_data(seed=1)
    _, g = o.loss_grad(p, X, T, w, bf16=False)
    pos = 0
    for out_, in_ in o.shapes:
        gw = g[pos:pos + out_ * in_]
        gb = g[pos + out_ * in_: pos + out_ * in_ + out_]
        assert np.abs(gw).max() > 0 and np.abs(gb).max() > 0
        pos += out_ * in_ + out_
    assert pos == p.size


def test_gelu_closed_forms():
    assert gelu(np.array(0.0)) == 0.0
    assert gelu_grad(np.array(0.0)) == pytest.approx(0.5, abs=1e-16)
    x = np.linspace(-6, 6, 101)
    # gelu(x) - gelu(-x) = x  (Phi(x) + Phi(-x) = 1)
    assert np.allclose(gelu(x) - gelu(-x), x, atol=1e-14)
    # Phi(1) = (1 + erf(1/sqrt 2)) / 2
    assert gelu(np.array(1.0)) == pytest.approx(0.5 * (1 + math.erf(1 / math.sqrt(2))), rel=1e-15)
    h = 1e-6
    assert np.allclose((gelu(x + h) - gelu(x - h)) / (2 * h), gelu_grad(x), atol=1e-8)
    assert gelu(np.array(40.0)) == 40.0 and abs(gelu(np.array(-40.0))) < 1e-300


def test_bf16_rounding_matches_a_library_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    x = np.concatenate([rng.normal(size=5000) * 10.0 ** rng.integers(-20, 20, 5000),
                        np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 0.0, 65504.0])])
    ref = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(bf16_round(x), ref)
    # ties to even: 1 + 2^-8 is halfway between 1 and 1 + 2^-7
    assert bf16_round(np.array([1.0 + 2 ** -8]))[0] == 1.0


def test_matrix_forward_equals_loop_forward():
    o, p, X, T, w = net_and_data(seed=2, width=5, depth=2, n_out=3, n=4)
    for bf16 in (False, True):
        Y, _ = o.forward(p, X, bf16)
        r = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
        layers = o.unpack(p)
        for s in range(X.shape[0]):
            h = [float(v) for v in r(X[s])]
            for q, (W, b) in enumerate(layers):
                Wr = r(W)
                z = [sum(Wr[j, i] * h[i] for i in range(len(h))) + b[j] for j in range(W.shape[0])]
                if q < len(layers) - 1:
                    h = [float(v) for v in r(gelu(np.array(z)))]
                else:
                    h = z
            assert np.allclose(h, Y[s], rtol=1e-13, atol=1e-13)


def test_zero_residual_gives_zero_loss_and_gradient():
    o, p, X, _, w = net_and_data(seed=4)
    Y, _ = o.forward(p, X, bf16=True)
    loss, g = o.loss_grad(p, X, Y, w, bf16=True)
    assert loss == 0.0 and not g.any()


def test_adam_step_against_its_closed_forms():
    """Adam's first step moves each parameter by lr * g / (|g| + eps) (the
    bias corrections undo the zero initial moments); with a constant
    gradient every later step does the same; with eps = 0 the step is
    invariant to scaling the gradient."""
    from oracle.mlp_oracle import adam_step
    rng = np.random.default_rng(5)
    p0 = rng.normal(size=50)
    g = rng.normal(size=50)
    z = np.zeros(50)
    lr = 1e-3
    p1, m1, v1 = adam_step(p0, g, z, z, 1, lr)
    assert np.allclose(p1 - p0, -lr * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    p, m, v = p1, m1, v1
    for t in range(2, 6):
        q, m, v = adam_step(p, g, m, v, t, lr)
        assert np.allclose(q - p, -lr * g / (np.abs(g) + 1e-8), rtol=1e-9, atol=0)
        p = q
    a, _, _ = adam_step(p0, g, z, z, 1, lr, eps=0.0)
    b, _, _ = adam_step(p0, 1e3 * g, z, z, 1, lr, eps=0.0)
    assert np.allclose(a, b, rtol=1e-14, atol=0)
    # two different gradients: the second step mixes them as the algorithm states
    g2 = rng.normal(size=50)
    q2, _, _ = adam_step(p1, g2, m1, v1, 2, lr)
    mh = (0.9 * 0.1 * g + 0.1 * g2) / (1 - 0.9 ** 2)
    vh = (0.999 * 0.001 * g * g + 0.001 * g2 * g2) / (1 - 0.999 ** 2)
    assert np.allclose(q2 - p1, -lr * mh / (np.sqrt(vh) + 1e-8), rtol=1e-12, atol=0)
