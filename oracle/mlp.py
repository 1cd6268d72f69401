"""FP64 reference of the learned inverse-CDF sampler (a 2-64-64-1 GELU network
standing in for the 2-D tables of §3.1 and §3.2; the paper has no learned
sampler).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain numpy: matrix
products, the chain rule written out, Adam.  The network, as the CUDA path
defines it:

  features   x1 = 2 (ln chi_c - ln chi_min) / (ln chi_max - ln chi_min) - 1,
             chi_c = chi clamped into the table's chi range;
             x2 = 2 u' - 1 with u' = U (QS) or u' = 2 min(U, 1 - U) (BW)
  layer 1    h1 = gelu(W1 x + b1)              (64)
  layer 2    h2 = gelu(W2 bf16(h1) + b2)       (64), bf16 = round to bfloat16
  layer 3    y  = W3 . h2 + b3
  output     QS: ln(xi / (1 - xi)) = y + 3 ln U + L(chi_c),  L(chi) = ln(chi / (1 + chi))
             BW: xi_s = min(1/2, 1 / (1 + exp(4 w(chi_c) y))),  w(chi) = sqrt(chi / (chi + 16/3)) / 2
             (xi_s is the electron's fraction if U <= 1/2, else the positron's;
             L and w centre and scale y: xi ~ U^3 as U -> 0 and grows with chi,
             the logit resolves 1 - xi at the hard end; the pair split narrows
             around 1/2 with width ~ sqrt(3 chi / 64) for small chi, where the
             BW map is 1/2 - w y to first order, and at large chi the folded
             split crowds towards 0, which its logit resolves)
  gelu(x)    = x/2 (1 + tanh(sqrt(2/pi) (x + 0.044715 x^3)))   (Hendrycks & Gimpel)
  loss       mean over the batch of (y - t)^2, with t the y whose output is xi*,
             xi* the reference sample of the same (chi, U)

Weights are used as bfloat16 (a master copy is kept in FP32 for Adam); the
rounding of h1 is treated as the identity in the backward pass.
Parameter vector layout (4417 floats): W1[64][2], b1[64], W2[64][64], b2[64],
W3[64], b3.
"""
from __future__ import annotations

import math

import numpy as np

H = 64
NPARAM = H * 2 + H + H * H + H + H + 1
C_GELU = math.sqrt(2.0 / math.pi)
A_GELU = 0.044715


def unpack(theta: np.ndarray):
    o = 0
    W1 = theta[o:o + 2 * H].reshape(H, 2); o += 2 * H
    b1 = theta[o:o + H]; o += H
    W2 = theta[o:o + H * H].reshape(H, H); o += H * H
    b2 = theta[o:o + H]; o += H
    W3 = theta[o:o + H]; o += H
    b3 = theta[o]
    return W1, b1, W2, b2, W3, b3


def bf16(a: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    nan = np.isnan(f)
    out[nan] = np.nan
    return out


def gelu(x):
    return 0.5 * x * (1.0 + np.tanh(C_GELU * (x + A_GELU * x ** 3)))


def gelu_grad(x):
    t = np.tanh(C_GELU * (x + A_GELU * x ** 3))
    return 0.5 * (1.0 + t) + 0.5 * x * (1.0 - t * t) * C_GELU * (1.0 + 3.0 * A_GELU * x * x)


def features(proc: int, chi, u, chi_min, chi_max):
    chi = np.asarray(chi, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    lc = np.log(np.clip(chi, chi_min, chi_max))
    x1 = 2.0 * (lc - math.log(chi_min)) / (math.log(chi_max) - math.log(chi_min)) - 1.0
    up = u if proc == 0 else 2.0 * np.minimum(u, 1.0 - u)
    return np.stack([x1, 2.0 * up - 1.0], axis=1)


def forward(theta, X, round_bf16=True):
    """Returns y and the cache for backward."""
    W1, b1, W2, b2, W3, b3 = unpack(np.asarray(theta, dtype=np.float64))
    if round_bf16:
        W1, W2, W3 = bf16(W1), bf16(W2), bf16(W3)
        b1, b2, b3 = bf16(b1), bf16(b2), float(bf16(np.array([b3]))[0])
    z1 = X @ W1.T + b1
    h1 = gelu(z1)
    h1q = bf16(h1) if round_bf16 else h1
    z2 = h1q @ W2.T + b2
    h2 = gelu(z2)
    y = h2 @ W3 + b3
    return y, (X, z1, h1q, z2, h2, W1, W2, W3)


def centre_scale(proc: int, chi, chi_min, chi_max):
    """L(chi_c) for QS, w(chi_c) for BW (the output map above)."""
    c = np.clip(np.asarray(chi, dtype=np.float64), chi_min, chi_max)
    if proc == 0:
        return np.log(c) - np.log1p(c)
    return 0.5 * np.sqrt(c / (c + 16.0 / 3.0))


def targets(proc: int, chi, u, xi, chi_min, chi_max):
    """t with output(t) = xi; for BW, xi is the electron's fraction."""
    u = np.asarray(u, dtype=np.float64)
    xi = np.asarray(xi, dtype=np.float64)
    cs = centre_scale(proc, chi, chi_min, chi_max)
    if proc == 0:
        return np.log(xi) - np.log1p(-xi) - 3.0 * np.log(u) - cs
    xs = np.where(u <= 0.5, xi, 1.0 - xi)  # folded fraction of the sampled lepton, in [0, 1/2]
    xs = np.clip(xs, 1e-300, 0.5)
    return np.log((1.0 - xs) / xs) / (4.0 * cs)


def loss_and_grad(theta, X, t, round_bf16=True):
    """Mean squared error and its gradient with respect to the parameter vector."""
    y, (X, z1, h1q, z2, h2, W1, W2, W3) = forward(theta, X, round_bf16)
    n = X.shape[0]
    r = y - t
    loss = float(np.mean(r * r))
    dy = 2.0 * r / n
    gW3 = h2.T @ dy
    gb3 = np.sum(dy)
    d2 = np.outer(dy, W3) * gelu_grad(z2)
    gW2 = d2.T @ h1q
    gb2 = np.sum(d2, axis=0)
    d1 = (d2 @ W2) * gelu_grad(z1)
    gW1 = d1.T @ X
    gb1 = np.sum(d1, axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, [gb3]])
    return loss, g


def output(proc: int, y, chi, u, chi_min, chi_max):
    """Sampled xi from the network output (the output map above): QS chi_gamma/chi,
    BW the folded fraction xi_s of the lepton that U selects."""
    u = np.asarray(u, dtype=np.float64)
    cs = centre_scale(proc, chi, chi_min, chi_max)
    if proc == 0:
        return 1.0 / (1.0 + np.exp(-(y + 3.0 * np.log(u) + cs)))
    return np.minimum(0.5, 1.0 / (1.0 + np.exp(4.0 * cs * np.asarray(y, dtype=np.float64))))


def adam(theta, m, v, g, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015), step counted from 1."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
