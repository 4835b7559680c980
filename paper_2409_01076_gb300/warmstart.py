"""Learned warm start: solver-generated training data, U-Net training, and the
time-to-steady comparison against the cold start.

1. `generate_dataset` runs many lid-driven cavities (U_lid = 0.1, Re log-uniform)
   to steady state with the batched SmrtLBM solver and keeps their (u, v, rho).
2. `train` fits the U-Net of unet.py (all arithmetic in libsmrt's NN kernels).
3. `time_to_steady` runs held-out cavities to the residual tolerance from rest
   (cold) and from the network's prediction (warm, f = f^eq(rho, u) of the
   prediction, bilinearly resampled when the lattice is not the training size).
   The plain solver stays the judge: the warm run must reach the same tolerance.

The network's output channels are u / U, v / U and (rho - 1) / (3 U^2).
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import workloads as W

U_LID = 0.1


def _S():
    import paper_2409_01076_gb300 as S
    return S


def sample_res(count: int, seed: int, lo: float = 100.0, hi: float = 10000.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.exp(rng.uniform(math.log(lo), math.log(hi), size=count)).tolist()


def generate_dataset(res, n: int = 256, tol: float = 1e-7, check_every: int = 1000, max_steps: int = 150000,
                     device: str = "cuda"):
    """Steady (or step-capped) cavities for each Re: returns (targets (len, n, n, 3) float32 CUDA, info)."""
    import torch
    S = _S()
    count = len(res)
    taus = [W.cavity_tau(n, U_LID, re) for re in res]
    b = S.smrt_batch_create([n] * count, [n] * count, taus, [U_LID] * count, W.CAVITY, S.SMRT_PREC_F32)
    t0 = time.perf_counter()
    S.smrt_batch_autotune(b, 6)
    S.smrt_batch_run(b, tol, check_every, max_steps, S.SMRT_BATCH_RESIDUAL_STRIDE)
    torch.cuda.synchronize()
    solve_s = time.perf_counter() - t0
    steps, resid, state = S.smrt_batch_status(b)
    targets = torch.empty((count, n, n, 3), dtype=torch.float32, device=device)
    rho = torch.empty((n, n), dtype=torch.float64, device=device)
    u = torch.empty((2, n, n), dtype=torch.float64, device=device)
    for k in range(count):
        S.smrt_batch_macros(b, k, rho, u)
        targets[k, ..., 0] = (u[0] / U_LID).float()
        targets[k, ..., 1] = (u[1] / U_LID).float()
        targets[k, ..., 2] = ((rho - 1.0) / (3 * U_LID * U_LID)).float()
    S.smrt_batch_destroy(b)
    info = {"count": count, "n": n, "solve_s": round(solve_s, 2), "node_updates": int(n * n * steps.sum()),
            "converged": int((state == S.SMRT_BATCH_CONVERGED).sum()),
            "capped": int((state == S.SMRT_BATCH_CAPPED).sum()),
            "diverged": int((state == S.SMRT_BATCH_DIVERGED).sum()),
            "steps_median": float(np.median(steps)), "steps_max": int(steps.max())}
    return targets, info


def train(net, res, targets, iters: int = 2000, batch: int = 16, lr: float = 1e-3, seed: int = 0,
          log_every: int = 100, warmup: int = 100, graph: bool = True):
    """Adam on random mini-batches: the learning rate rises linearly over the first `warmup`
    iterations, under a cosine decay over all of them.  Returns the loss history and the seconds.

    Measured on 256 solver-generated 256^2 cavities (800 iterations, two seeds, both GEMM
    backends): a peak rate of 1e-3 reaches a held-out MSE of 0.7-1.3e-4 in every run, with or
    without the warm-up; 2e-3 is unstable (loss spikes when the rate peaks, stalls near the
    mean-field loss in some runs).

    graph: the forward and backward pass is recorded once as a CUDA graph (UNet.capture) and
    replayed on static input tensors that each iteration's batch is copied into; Adam runs outside
    the graph (its step-dependent scalars change every iteration)."""
    import torch
    from .unet import input_grid
    rng = np.random.Generator(np.random.PCG64(seed))
    n = targets.shape[1]
    count = len(res)
    hist = []
    xs = ts = None
    t0 = time.perf_counter()
    for it in range(iters):
        idx = rng.choice(count, size=min(batch, count), replace=False)
        x = input_grid([res[i] for i in idx], n, n)
        tgt = targets[torch.as_tensor(idx, device=targets.device)].contiguous()
        cur = lr * min(1.0, (it + 1) / max(warmup, 1)) * 0.5 * (1.0 + math.cos(math.pi * it / iters))
        if graph:
            if xs is None:
                xs, ts = x.clone(), tgt.clone()
            else:
                xs.copy_(x)
                ts.copy_(tgt)
            if net._graph is None or net._graph_in[0] is not xs:
                net.capture(xs, ts)         # first iteration, or after the loss scale changed
            net.replay()
        else:
            net.loss_and_grad(x, tgt)
        net.adam_step(cur)
        if it % log_every == 0 or it == iters - 1:
            hist.append((it, float(net._loss.item())))
    torch.cuda.synchronize()
    return hist, time.perf_counter() - t0


def predict_fields(net, res, n: int, train_n: int = 256):
    """Network prediction for each Re at the training size, resampled to n x n: returns
    (rho (len, n, n) float64, u (len, 2, n, n) float64) in lattice units."""
    import torch
    from . import nn as K
    from .unet import input_grid
    x = input_grid(list(res), train_n, train_n)
    y = net.predict(x)
    if n != train_n:
        z = torch.empty((len(res), n, n, 3), dtype=torch.float32, device=y.device)
        K.smrt_nn_resize_bilinear(y, z)
        y = z
    yd = y.double()
    rho = 1.0 + 3 * U_LID * U_LID * yd[..., 2]
    u = torch.stack([U_LID * yd[..., 0], U_LID * yd[..., 1]], dim=1)
    return rho.contiguous(), u.contiguous()


def time_to_steady(res, n: int, net=None, tol: float = 1e-7, check_every: int = 1000, max_steps: int = 400000,
                   train_n: int = 256):
    """Runs one batch of n x n cavities (one per Re) to the tolerance, cold (net None) or warm from the
    network evaluated at its training size train_n.
    Returns per-cavity steps and states, the wall time of the whole batch and of the prediction."""
    import torch
    S = _S()
    count = len(res)
    taus = [W.cavity_tau(n, U_LID, re) for re in res]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b = S.smrt_batch_create([n] * count, [n] * count, taus, [U_LID] * count, W.CAVITY, S.SMRT_PREC_F32)
    t_pred = 0.0
    if net is not None:
        tp = time.perf_counter()
        rho, u = predict_fields(net, res, n, train_n)
        for k in range(count):
            S.smrt_batch_init_macros(b, k, rho[k], u[k])
        torch.cuda.synchronize()
        t_pred = time.perf_counter() - tp
    S.smrt_batch_run(b, tol, check_every, max_steps, S.SMRT_BATCH_RESIDUAL_STRIDE)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    steps, resid, state = S.smrt_batch_status(b)
    fields = []
    rho_k = torch.empty((n, n), dtype=torch.float64, device="cuda")
    u_k = torch.empty((2, n, n), dtype=torch.float64, device="cuda")
    for k in range(count):
        S.smrt_batch_macros(b, k, rho_k, u_k)
        fields.append(u_k.clone())
    S.smrt_batch_destroy(b)
    return {"steps": steps.tolist(), "state": state.tolist(), "residual": resid.tolist(), "wall_s": wall,
            "predict_s": t_pred}, fields
