"""Plain FP64 oracle of the surface-charge surrogate (a multilayer
perceptron with GELU hidden layers and a mean-squared-error loss).

TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the tests import it; the CUDA
library never does, and this module imports nothing of the CUDA package.

The paper (Sun et al., arXiv 2303.14119) has no surrogate: what is checked
here is the textbook network and its backpropagation, written out with numpy
matrix products in FP64:

  H_0 = X,  Z_l = H_l W_l^T + b_l,  H_{l+1} = gelu(Z_l)   (hidden layers)
  Y = H_L W_out^T + b_out
  loss = (1/n) sum_samples sum_outputs w_o (Y - T)^2
  gelu(z) = z Phi(z) = z (1 + erf(z / sqrt 2)) / 2,  gelu'(z) = Phi(z) + z phi(z)

Parameters are one flat vector, layer by layer: W_l [out][in] row-major,
then b_l [out].  With bf16=True the oracle also rounds, to bf16 (through
FP32, round to nearest even), exactly the values the tensor-core kernels
hold in bf16: the inputs, the weights, the hidden activations, the output
gradient dL/dY and the pre-activation gradients; everything else stays FP64.
"""
from __future__ import annotations

import math

import numpy as np

try:
    from scipy.special import erf as _erf
except ImportError:  # pragma: no cover - scipy is in both images
    _erf = np.vectorize(math.erf)


def bf16_round(x):
    """Round to bf16 through FP32 (round to nearest, ties to even); finite
    inputs.  Returns FP64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = (u + np.uint64(0x7FFF) + ((u >> np.uint64(16)) & np.uint64(1))) >> np.uint64(16)
    return (r << np.uint64(16)).astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


class MLPOracle:
    def __init__(self, n_in: int, width: int, depth: int, n_out: int):
        self.dims = [n_in] + [width] * depth + [n_out]
        self.shapes = [(self.dims[q + 1], self.dims[q]) for q in range(len(self.dims) - 1)]

    def param_count(self) -> int:
        return sum(o * i + o for o, i in self.shapes)

    def unpack(self, params):
        params = np.asarray(params, dtype=np.float64)
        out, p = [], 0
        for o, i in self.shapes:
            W = params[p:p + o * i].reshape(o, i)
            p += o * i
            b = params[p:p + o]
            p += o
            out.append((W, b))
        assert p == params.size
        return out

    def forward(self, params, X, bf16=True):
        """Outputs Y [n][n_out] and the cache for backward."""
        r = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
        layers = self.unpack(params)
        H = r(np.asarray(X, dtype=np.float64))
        hs, zs, ws = [H], [], []
        for q, (W, b) in enumerate(layers):
            Wr = r(W)
            ws.append(Wr)
            Z = H @ Wr.T + b
            if q == len(layers) - 1:
                return Z, (hs, zs, ws)
            zs.append(Z)
            H = r(gelu(Z))
            hs.append(H)
        raise AssertionError("unreachable")

    def loss(self, params, X, T, w=None, bf16=True):
        Y, _ = self.forward(params, X, bf16)
        w = np.ones(Y.shape[1]) if w is None else np.asarray(w, dtype=np.float64)
        return float(((Y - T) ** 2 * w).sum() / Y.shape[0])

    def loss_grad(self, params, X, T, w=None, bf16=True):
        """(loss, flat gradient) by backpropagation."""
        r = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
        Y, (hs, zs, ws) = self.forward(params, X, bf16)
        n = Y.shape[0]
        w = np.ones(Y.shape[1]) if w is None else np.asarray(w, dtype=np.float64)
        loss = float(((Y - T) ** 2 * w).sum() / n)
        dZ = r(2.0 * w * (Y - T) / n)  # dL/dY
        grads = []
        L = len(ws)
        for q in range(L - 1, -1, -1):
            dW = dZ.T @ hs[q]
            db = dZ.sum(axis=0)
            grads.append((dW, db))
            if q > 0:
                dZ = r((dZ @ ws[q]) * gelu_grad(zs[q - 1]))
        grads.reverse()
        flat = np.concatenate([np.concatenate([dW.ravel(), db]) for dW, db in grads])
        return loss, flat


def adam_step(p, g, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One step of Adam (Kingma and Ba, "Adam: A method for stochastic
    optimization", ICLR 2015, Algorithm 1) in FP64: the moment estimates
    m <- beta1 m + (1 - beta1) g and v <- beta2 v + (1 - beta2) g^2, their
    bias corrections by 1 - beta^t, and p <- p - lr mhat / (sqrt(vhat) + eps).
    t counts steps from 1.  Returns (p, m, v) as new arrays."""
    p, g, m, v = (np.asarray(a, dtype=np.float64) for a in (p, g, m, v))
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v
