"""CPU oracle for the learned warm start of the lead surface Green's function.
TEST INFRASTRUCTURE ONLY: only the tests, the smoke check and the benchmark's CPU
leg may import it; the library never does, and it shares no code with the CUDA path.

The network has no counterpart in the paper (the paper's own machine learning
predicts Hamiltonians, Sec. IV); it is the learned initial guess g0 for the
guess-driven open-boundary solver.  What it computes, in plain numpy float64:

  features   x = [ sqrt(b) Re diag(H00)            (b)
                 | sqrt(b) Re H00[i,j], i < j        (b(b-1)/2, row-major)
                 | sqrt(b) Im H00[i,j], i < j        (b(b-1)/2)
                 | sqrt(b) Re H01                    (b^2, row-major)
                 | sqrt(b) Im H01                    (b^2)
                 | E / 3
                 | sin(w_m E), cos(w_m E), m = 0..31 ]  -> K0 = 3 b^2 + 65 values,
             zero-padded to K0P (a multiple of 128); w_m = 2^(m/4), written as
             2^(m div 4) times 2^((m mod 4)/4) so that both sides form the same double
             (a Fourier encoding of the energy, finer than one BF16 feature resolves);
  network    z1 = W1 x + c1,  h1 = relu(z1)           (hidden)
             z2 = W2 h1 + c2, h2 = relu(z2)           (hidden)
             y  = W3 h2 + c3                          (2 b^2)
  output     g0 = y[:b^2] + i y[b^2:]  (row-major b x b);
  loss       L = sum (y - t)^2 / (n * 2 b^2) over a batch of n samples, with t the
             packed Sancho-Rubio surface function;
  optimiser  Adam (Kingma & Ba 2015) with bias correction.

The weights are BF16 and the accumulation FP32 on the GPU.  With ``quant=True`` the
oracle rounds to BF16 exactly the values the GPU feeds its tensor-core products
(features, weights, hidden activations and back-propagated signals) and computes
everything else in float64; the parity tests compare against that.  All functions
are pinned by the oracle tests (finite differences for the gradients, closed forms
for the rounding, the first Adam step and the packing).
"""
from __future__ import annotations

import numpy as np

__all__ = ["bf16_round", "mlp_dims", "param_layout", "split_params", "pack_features", "pack_target",
           "unpack_output", "forward", "loss_and_grads", "adam_step"]

E_SCALE = 1.0 / 3.0
N_FREQ = 32
_ROOTS2 = (1.0, 1.189207115002721, 1.4142135623730951, 1.6817928305074290)   # 2^(k/4), k = 0..3


def freqs():
    """w_m = 2^(m/4), m = 0..N_FREQ-1, as 2^(m div 4) * 2^((m mod 4)/4)."""
    return np.array([np.ldexp(_ROOTS2[m & 3], m >> 2) for m in range(N_FREQ)])


def bf16_round(x):
    """Round float64 values to the nearest BF16 value (8 significant bits), ties to
    even, in one rounding step.  Exact for normal values in the BF16 range."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)                   # x = m 2^e, 0.5 <= |m| < 1
    return np.ldexp(np.rint(np.ldexp(m, 8)), e - 8)   # rint rounds ties to even


def mlp_dims(b, hidden=512):
    """(K0, K0P, hidden, NOUT): feature count, padded feature count, width, outputs."""
    k0 = 3 * b * b + 1 + 2 * N_FREQ
    k0p = (k0 + 127) // 128 * 128
    return k0, k0p, hidden, 2 * b * b


def param_layout(b, hidden=512):
    """Offsets of W1 [hidden][K0P], c1 [hidden], W2 [hidden][hidden], c2 [hidden],
    W3 [NOUT][hidden], c3 [NOUT] in one flat parameter vector, and its length."""
    _, k0p, h, nout = mlp_dims(b, hidden)
    sizes = [("W1", h * k0p), ("c1", h), ("W2", h * h), ("c2", h), ("W3", nout * h), ("c3", nout)]
    off, out = 0, {}
    for name, n in sizes:
        out[name] = (off, n)
        off += n
    return out, off


def split_params(theta, b, hidden=512):
    """Views of the flat parameter vector as the six arrays."""
    _, k0p, h, nout = mlp_dims(b, hidden)
    lay, _ = param_layout(b, hidden)
    shapes = {"W1": (h, k0p), "c1": (h,), "W2": (h, h), "c2": (h,), "W3": (nout, h), "c3": (nout,)}
    return {k: theta[o:o + n].reshape(shapes[k]) for k, (o, n) in lay.items()}


def pack_features(H00, H01, E):
    """Feature vector of one (lead, energy) sample, zero-padded to K0P (see header)."""
    b = H00.shape[0]
    k0, k0p, _, _ = mlp_dims(b)
    s = np.sqrt(float(b))
    iu = np.triu_indices(b, 1)
    parts = [H00.real[np.arange(b), np.arange(b)], H00.real[iu], H00.imag[iu],
             H01.real.reshape(-1), H01.imag.reshape(-1)]
    x = np.zeros(k0p)
    nh = 3 * b * b
    x[:nh] = np.concatenate(parts) * s
    x[nh] = E * E_SCALE
    w = freqs() * E
    x[nh + 1:nh + 1 + 2 * N_FREQ:2] = np.sin(w)
    x[nh + 2:nh + 2 + 2 * N_FREQ:2] = np.cos(w)
    return x


def unpack_features(x, b):
    """Inverse of the packing (for the pins): (H00, H01, E)."""
    s = np.sqrt(float(b))
    nh = 3 * b * b
    v = x[:nh] / s
    nu = b * (b - 1) // 2
    d, re, im = v[:b], v[b:b + nu], v[b + nu:b + 2 * nu]
    H00 = np.zeros((b, b), dtype=np.complex128)
    iu = np.triu_indices(b, 1)
    H00[iu] = re + 1j * im
    H00 = H00 + H00.conj().T
    H00[np.arange(b), np.arange(b)] = d
    r = v[b + 2 * nu:]
    H01 = (r[:b * b] + 1j * r[b * b:]).reshape(b, b)
    return H00, H01, x[nh] / E_SCALE


def pack_target(g):
    """t = [Re g | Im g] (row-major), the regression target of one sample."""
    return np.concatenate([g.real.reshape(-1), g.imag.reshape(-1)])


def unpack_output(y, b):
    """g0 = y[:b^2] + i y[b^2:] reshaped to b x b."""
    return (y[:b * b] + 1j * y[b * b:2 * b * b]).reshape(b, b)


def _q(x, quant):
    return bf16_round(x) if quant else x


def forward(theta, X, b, hidden=512, quant=True):
    """Network outputs Y [n][NOUT] for features X [n][K0P] and the intermediates."""
    p = split_params(theta, b, hidden)
    Xq = _q(X, quant)
    W1, W2, W3 = (_q(p[k], quant) for k in ("W1", "W2", "W3"))
    z1 = Xq @ W1.T + p["c1"]
    h1 = _q(np.maximum(z1, 0.0), quant)
    z2 = h1 @ W2.T + p["c2"]
    h2 = _q(np.maximum(z2, 0.0), quant)
    Y = h2 @ W3.T + p["c3"]
    return Y, dict(Xq=Xq, W1=W1, W2=W2, W3=W3, z1=z1, h1=h1, z2=z2, h2=h2)


def loss_and_grads(theta, X, T, b, hidden=512, quant=True):
    """Mean squared error and its gradient with respect to the flat parameters.

    Backward pass (chain rule, relu'(z) = [z > 0]):
      dY  = 2 (Y - T) / (n NOUT)
      dW3 = dY^T h2,   dc3 = sum_rows dY,   dh2 = dY W3
      dz2 = dh2 [z2 > 0], dW2 = dz2^T h1, dc2 = sum_rows dz2, dh1 = dz2 W2
      dz1 = dh1 [z1 > 0], dW1 = dz1^T x,  dc1 = sum_rows dz1.
    With ``quant`` the operands of the products (dY, dz2, dz1 where they enter a
    product) are rounded to BF16 like the GPU's; the bias sums use the unrounded values."""
    n = X.shape[0]
    _, _, _, nout = mlp_dims(b, hidden)
    Y, c = forward(theta, X, b, hidden, quant)
    R = Y - T
    loss = float(np.sum(R * R) / (n * nout))
    dY = 2.0 * R / (n * nout)
    dYq = _q(dY, quant)
    g = {}
    g["W3"] = dYq.T @ c["h2"]
    g["c3"] = dY.sum(axis=0)
    dh2 = dYq @ c["W3"]
    dz2 = dh2 * (c["z2"] > 0)
    dz2q = _q(dz2, quant)
    g["W2"] = dz2q.T @ c["h1"]
    g["c2"] = dz2.sum(axis=0)
    dh1 = dz2q @ c["W2"]
    dz1 = dh1 * (c["z1"] > 0)
    dz1q = _q(dz1, quant)
    g["W1"] = dz1q.T @ c["Xq"]
    g["c1"] = dz1.sum(axis=0)
    lay, total = param_layout(b, hidden)
    grad = np.zeros(total)
    for k, (o, m) in lay.items():
        grad[o:o + m] = g[k].reshape(-1)
    return loss, grad, Y


def adam_step(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step index t >= 1):
      m = beta1 m + (1 - beta1) g,  v = beta2 v + (1 - beta2) g^2,
      theta -= lr * (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
