"""FP64 numpy oracle of the surrogate MLP (GELU hidden layers, linear output,
mean squared error, Adam).

TEST INFRASTRUCTURE ONLY: it checks the library's tensor-core training and
inference kernels; the library never calls it.  Parameters are one vector:
for each layer W [N][K] (row-major) then b [N].

With ``bf16=True`` the forward and backward passes round, like the tensor-core
path, the weights, the inputs, the hidden activations and the back-propagated
pre-activation gradients to bfloat16 (round to nearest even) before each
product, and keep everything else in FP64.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf


def bf16_round(a):
    """Round float64 values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    out = rounded.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    if nan.any():
        out[nan] = np.nan
    return out


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


class MLPOracle:
    def __init__(self, dims):
        self.dims = list(dims)
        self.L = len(dims) - 1
        self.offsets = []
        o = 0
        for l in range(self.L):
            K, N = dims[l], dims[l + 1]
            self.offsets.append((o, o + N * K, o + N * K + N, N, K))
            o += N * K + N
        self.n_params = o

    def unpack(self, p):
        return [(p[a:b].reshape(N, K), p[b:c]) for a, b, c, N, K in self.offsets]

    def init_params(self, rng):
        p = np.zeros(self.n_params)
        for (a, b, c, N, K) in self.offsets:
            p[a:b] = rng.normal(0.0, np.sqrt(2.0 / K), N * K)  # He initialisation
        return p

    def forward(self, p, x, bf16=False):
        r = bf16_round if bf16 else (lambda v: v)
        acts, zs = [r(np.asarray(x, np.float64))], []
        h = acts[0]
        for l, (W, b) in enumerate(self.unpack(p)):
            z = h @ r(W).T + b
            if l < self.L - 1:
                zs.append(z)
                h = r(gelu(z))
                acts.append(h)
            else:
                return z, acts, zs

    def loss_and_grad(self, p, x, t, bf16=False):
        """MSE loss mean((y - t)^2) and its gradient with respect to p."""
        r = bf16_round if bf16 else (lambda v: v)
        y, acts, zs = self.forward(p, x, bf16)
        B, N = y.shape
        loss = np.mean((y - t) ** 2)
        dz = r(2.0 * (y - t) / (B * N))
        g = np.zeros_like(p)
        layers = self.unpack(p)
        for l in range(self.L - 1, -1, -1):
            a, bo, c, Nl, Kl = self.offsets[l]
            g[a:bo] = (dz.T @ acts[l]).ravel()
            g[bo:c] = dz.sum(0)
            if l > 0:
                W = r(layers[l][0])
                dz = r((dz @ W) * gelu_grad(zs[l - 1]))
        return loss, g

    @staticmethod
    def adam(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        p = p - lr * (m / (1 - b1 ** t)) / (np.sqrt(v / (1 - b2 ** t)) + eps)
        return p, m, v


def ensemble_stats(ys, scale=None, shift=None, n_spread=0, tol=0.0, row=None, n_row=0, offset=None):
    """Ensemble statistics by their definitions, in FP64: members' outputs
    mapped to z = (y * scale + shift) * row_b + offset (row_b, one factor per
    batch row, on the first n_row outputs only), mean and population standard
    deviation over the members, spread = max of the std over the first
    n_spread outputs, fallback = spread > tol.  ys: sequence of [B][n_out]."""
    Z = np.stack([np.asarray(y, np.float64) for y in ys])
    if scale is not None:
        Z = Z * np.asarray(scale, np.float64) + np.asarray(shift, np.float64)
    if row is not None:
        Z[:, :, :n_row] *= np.asarray(row, np.float64)[None, :, None]
    if offset is not None:
        Z = Z + np.asarray(offset, np.float64)
    mean = Z.sum(0) / len(ys)
    std = np.sqrt(((Z - mean) ** 2).sum(0) / len(ys))
    spread = std[:, :n_spread].max(1) if n_spread > 0 else np.zeros(len(mean))
    return mean, std, spread, spread > tol
