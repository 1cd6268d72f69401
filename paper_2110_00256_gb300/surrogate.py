"""Training and evaluation of the learned inverse-CDF sampler on the GPU.

Training data: (chi, U, xi) with chi log-uniform over the table range (drawn
as `rows` distinct values, each with its share of the draws), U uniform in
(0, 1), and xi the exact inverse CDF of the same (chi, U) computed on the GPU
(qed_exact_sample: FP64 quadrature of the spectra, no table).  Every step of
the training runs in libqed's kernels (forward, backward, Adam).
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import api


def chi_range(tables: api.Tables, proc: int):
    p = tables.params
    ax = p.qs if proc == api.QED_PROC_QS else p.bw
    return ax.chi_min, ax.chi_max


def make_data(tables: api.Tables, proc: int, n: int, seed: int, rows: int = 16384, device="cuda"):
    """n training samples (chi, U, xi) on the device, xi from the exact inverse
    CDF; chi takes `rows` log-uniform values (n // rows draws each), shuffled."""
    lo, hi = (math.log(v) for v in chi_range(tables, proc))
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    rows = max(1, min(rows, n))
    k = max(1, n // rows)
    chi_rows = torch.exp(lo + (hi - lo) * torch.rand(rows, generator=g, device=device, dtype=torch.float64))
    u = torch.rand(rows * k, generator=g, device=device, dtype=torch.float64).clamp_(1e-15, 1.0 - 1e-15)
    # sorted within each chi row: neighbouring threads of the exact sampler then
    # take neighbouring intervals (similar work)
    u = torch.sort(u.view(rows, k), dim=1).values.reshape(-1)
    xi = api.qed_exact_sample(proc, chi_rows, u)
    chi = chi_rows.repeat_interleave(k)
    perm = torch.randperm(rows * k, generator=g, device=device)
    return chi[perm], u[perm], xi[perm]


def train(mlp: api.Mlp, data_tables: api.Tables, proc: int, n_samples: int = 10_000_000, epochs: int | None = None,
          batch: int = 4096, lr: float = 4e-3, lr_final: float = 1e-4, seed: int = 1, log_every: int = 0):
    """Train one network on n_samples exact samples (epochs passes, Adam with a
    cosine decay of the step size from lr to lr_final); returns the loss history
    (one value per logged step) and timings.  The defaults, 48 epochs of 4096
    (1.2e5 steps) for photon emission and 96 (2.3e5 steps) for the pair split,
    put every chi bin's KS distance to the exact distribution below 1e-3; 8
    epochs of 16384 (5e3 steps) had left the pair-split network's worst bin
    near 7e-3: the accuracy follows the number of steps."""
    if epochs is None:
        epochs = 48 if proc == api.QED_PROC_QS else 96
    t_data = time.perf_counter()
    chi, u, xi = make_data(data_tables, proc, n_samples, seed)
    n_samples = chi.numel()  # (a whole number of draws per chi value)
    torch.cuda.synchronize()
    data_s = time.perf_counter() - t_data
    g = torch.Generator(device=chi.device)
    g.manual_seed(seed + 1)
    steps = epochs * ((n_samples + batch - 1) // batch)
    loss = torch.zeros(1, dtype=torch.float32, device=chi.device)
    hist = []
    k = 0
    t0 = time.perf_counter()
    for ep in range(epochs):
        perm = torch.randperm(n_samples, generator=g, device=chi.device)
        c, uu, x = chi[perm], u[perm], xi[perm]
        for b in range(0, n_samples, batch):
            e = min(b + batch, n_samples)
            # cosine decay from lr to lr_final
            rate = lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * k / max(steps - 1, 1)))
            mlp.train_step(proc, c[b:e], uu[b:e], x[b:e], rate, loss)
            k += 1
            if log_every and k % log_every == 0:
                hist.append(float(loss.item()))
    torch.cuda.synchronize()
    return {"steps": k, "seconds": time.perf_counter() - t0, "data_seconds": data_s, "final_loss": float(loss.item()),
            "history": hist}


def ks_distance(a: torch.Tensor, b: torch.Tensor) -> float:
    """Two-sample Kolmogorov-Smirnov distance between two sets of samples."""
    x = torch.sort(a.double()).values
    y = torch.sort(b.double()).values
    allv = torch.cat([x, y])
    fa = torch.searchsorted(x, allv, right=True).double() / x.numel()
    fb = torch.searchsorted(y, allv, right=True).double() / y.numel()
    return float((fa - fb).abs().max().item())


def compare(sampler, tables: api.Tables, proc: int, n: int = 1_000_000, seed: int = 99, bins: int = 5,
            rows: int = 2000):
    """KS distance between a sampler's xi and the exact inverse CDF's on the
    same (chi, U), overall and in `bins` equal log-chi bins of the table range.
    `sampler(chi, u)` returns xi on the device (QS chi_gamma/chi, BW the
    electron's fraction)."""
    lo, hi = (math.log(v) for v in chi_range(tables, proc))
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    k = max(1, n // rows)
    t = (torch.arange(rows, device="cuda", dtype=torch.float64) + torch.rand(rows, generator=g, device="cuda",
                                                                             dtype=torch.float64)) / rows
    chi_rows = torch.exp(lo + (hi - lo) * t)
    u = torch.rand(rows * k, generator=g, device="cuda", dtype=torch.float64).clamp_(1e-15, 1.0 - 1e-15)
    xe = api.qed_exact_sample(proc, chi_rows, u)
    chi = chi_rows.repeat_interleave(k)
    xs = sampler(chi, u)
    key = (lambda v: torch.log(v)) if proc == api.QED_PROC_QS else (lambda v: v)
    out = {"overall": ks_distance(key(xs), key(xe)), "bins": []}
    tt = t.repeat_interleave(k)
    for i in range(bins):
        m = (tt >= i / bins) & (tt < (i + 1) / bins)
        out["bins"].append(ks_distance(key(xs[m]), key(xe[m])))
    return out


def compare_tables(ta: api.Tables, prec_a: int, tb: api.Tables, prec_b: int, proc: int, n: int = 1_000_000,
                   seed: int = 98) -> float:
    """KS distance between the samples of two table sets on the same (chi, U)."""
    p = tb.params
    ax = p.qs if proc == api.QED_PROC_QS else p.bw
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    lo, hi = math.log(ax.chi_min), math.log(ax.chi_max)
    chi = torch.exp(lo + (hi - lo) * torch.rand(n, generator=g, device="cuda", dtype=torch.float64))
    u = torch.rand(n, generator=g, device="cuda", dtype=torch.float64).clamp_(1e-15, 1.0 - 1e-15)
    a = api.qed_table_sample(ta, proc, prec_a, chi, u)
    b = api.qed_table_sample(tb, proc, prec_b, chi, u)
    key = (lambda v: torch.log(v)) if proc == api.QED_PROC_QS else (lambda v: v)
    return ks_distance(key(a), key(b))
