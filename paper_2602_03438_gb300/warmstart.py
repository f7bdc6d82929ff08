"""Learned warm start of the lead surface Green's function (include/negf_warmstart.h):
training pairs from the plain solver, training on the GPU, and the guess-driven OBC.

This module only sequences libnegf calls and moves tensors; every arithmetic step
(decimation, Newton, retarded-root test, feature packing, network forward and
backward, Adam) runs in the library's kernels.  The leads are semi-infinite chains
of the block pair (H00, H01) facing +x; each one is posed to negf_obc as the right
lead of a two-block device [H00, H00] with hop H01.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import negf as N


def lead_system(H00: np.ndarray, H01: np.ndarray, lead: np.ndarray, E: np.ndarray, eta: float,
                device="cuda") -> N.System:
    """One nb = 2 device per lead that has samples, energies in sample order.  The
    samples must be grouped by lead in increasing lead order (e.g. np.repeat)."""
    lead = np.asarray(lead)
    if lead.size and np.any(np.diff(lead) < 0):
        raise ValueError("samples must be grouped by lead in increasing order")
    uniq, counts = np.unique(lead, return_counts=True)
    b = H00.shape[-1]
    Hd = np.stack([np.stack([H00[l], H00[l]]) for l in uniq])
    Hu = np.stack([H01[l] for l in uniq])
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).to(device)
    return N.System([2] * len(uniq), [b] * len(uniq), [int(c) for c in counts], t(Hd), t(Hu), None, None,
                    t(np.asarray(E, dtype=np.float64)), float(eta))


@dataclass
class ObcResult:
    gs_R: torch.Tensor      # [n][b][b] right-lead surface functions
    sigma_R: torch.Tensor
    iters: np.ndarray       # [n][2] decimation steps (L, R)
    newton: np.ndarray      # [n][2] Newton steps (L, R)
    status: np.ndarray      # [n]
    ms: float               # device time of the negf_obc call (CUDA events)


def solve_surfaces(ctx: N.Context, sys: N.System, g0_R=None, g0_L=None, stream=None) -> ObcResult:
    """negf_obc over the lead batch, optionally warm-started, timed with CUDA events."""
    n = int(sum(sys.ne))
    b = sys.bs[0]
    dev = sys.energy.device
    z = lambda: torch.empty(n * b * b, dtype=torch.complex128, device=dev)
    sL, sR, gsR = z(), z(), z()
    iters = torch.zeros(2 * n, dtype=torch.int32, device=dev)
    newton = torch.zeros_like(iters)
    status = torch.zeros(n, dtype=torch.int32, device=dev)
    s = stream or torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    N.negf_obc(ctx, sys, sL, sR, iters, status, g0_L=g0_L, g0_R=g0_R, gs_R=gsR, newton=newton, stream=s)
    e1.record(s)
    ctx.check(ctx.sync(s))
    return ObcResult(gsR.view(n, b, b), sR.view(n, b, b), iters.cpu().numpy().reshape(n, 2),
                     newton.cpu().numpy().reshape(n, 2), status.cpu().numpy(), e0.elapsed_time(e1))


@dataclass
class Network:
    dims: N.MlpDims
    params: torch.Tensor
    losses: list


def train_network(ctx: N.Context, b: int, X: torch.Tensor, G: torch.Tensor, n: int, theta0: np.ndarray,
                  steps: int = 2000, batch: int = 256, lr: float = 1e-3, seed: int = 0, hidden: int = 512,
                  log_every: int = 100) -> Network:
    """Adam on minibatches drawn (seeded, host side) from the n training pairs (X from
    negf_mlp_pack, G the surface functions); the learning rate drops 10x for the last
    fifth of the steps.  Returns the trained parameters and the logged losses."""
    dims = N.negf_mlp_get_dims(b, hidden)
    dev = X.device
    params = torch.from_numpy(np.ascontiguousarray(theta0, dtype=np.float32)).to(dev)
    m = torch.zeros(dims.n_params, dtype=torch.float32, device=dev)
    v, grad = torch.zeros_like(m), torch.zeros_like(m)
    loss = torch.zeros(1, dtype=torch.float64, device=dev)
    rng = np.random.default_rng(seed)
    rows = torch.from_numpy(np.stack([rng.choice(n, size=batch, replace=False) for _ in range(steps)])
                            .astype(np.int32)).to(dev)
    hist = []
    for k in range(steps):
        step_lr = lr if k < 0.8 * steps else 0.1 * lr
        N.negf_mlp_train_step(ctx, dims, params, m, v, grad, k + 1, step_lr, batch, X, G, loss, update=True,
                              rows=rows[k], n_set=n)
        if (k + 1) % log_every == 0 or k == 0:
            hist.append((k + 1, float(loss.item())))
    ctx.check(ctx.sync())
    return Network(dims, params, hist)


def predict(ctx: N.Context, net: Network, H00: np.ndarray, H01: np.ndarray, lead: np.ndarray,
            E: np.ndarray, stream=None):
    """Network guesses g0 [n][b][b] for the samples, with the device time of packing +
    inference (ms)."""
    dev = net.params.device
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    H00d, H01d, leadd, Ed = t(H00), t(H01), t(np.asarray(lead, np.int32)), t(np.asarray(E, np.float64))
    s = stream or torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    X = N.negf_mlp_pack(ctx, net.dims.b, H00d, H01d, leadd, Ed, stream=s)
    g0 = N.negf_mlp_forward(ctx, net.dims, net.params, len(lead), X, stream=s)
    e1.record(s)
    ctx.check(ctx.sync(s))
    return g0, e0.elapsed_time(e1)
