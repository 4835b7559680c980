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
            "steps_median": float(np.median(steps)), "steps_max": int(steps.max()),
            "residual_quantiles": {q: float(np.quantile(resid, v)) for q, v in
                                   (("p50", 0.5), ("p90", 0.9), ("p99", 0.99), ("max", 1.0))}}
    capped = resid[state == S.SMRT_BATCH_CAPPED]
    if capped.size:
        info["capped_residual_median"] = float(np.median(capped))
        info["capped_re_min"] = float(min(re for re, st in zip(res, state) if st == S.SMRT_BATCH_CAPPED))
    return targets, info


def train(net, res, targets, iters: int = 2000, batch: int = 16, lr: float = 1e-3, seed: int = 0,
          log_every: int = 100, warmup: int = 100, graph: bool = True):
    """Adam on random mini-batches: the learning rate rises linearly over the first `warmup`
    iterations, under a cosine decay over all of them.  Returns the loss history and the seconds.

    Measured on 256 solver-generated 256^2 cavities (800 iterations, two seeds, both GEMM
    backends): a peak rate of 1e-3 reaches a held-out MSE of 0.7-1.3e-4 in every run, with or
    without the warm-up; 2e-3 is unstable (loss spikes when the rate peaks, stalls near the
    mean-field loss in some runs).  On 2,000 cavities the held-out error keeps falling with the
    length of the schedule: max |u - u_steady| / U over nine steady cavities (Re 130-2,500) of
    0.08-0.15 after 2,000 iterations, 0.024-0.032 after 6,000 and 0.010-0.017 after 12,000 (rms
    2.5e-3 -> 1.0e-3 -> 5e-4 at Re <= 1,200); 7e-4 instead of 1e-3 at 6,000 was worse.

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


def _u_of(h, n):
    import torch
    S = _S()
    rho = torch.empty((n, n), dtype=torch.float64, device="cuda")
    u = torch.empty((2, n, n), dtype=torch.float64, device="cuda")
    S.smrt_macros(h, rho, u)
    return u


class _Tracked:
    """One cavity advanced in chunks of K updates on its own handle; after each chunk the stride
    residual r = ||u(t) - u(t-K)|| / (K ||u(t)||) over all nodes.  Step time is taken with CUDA events
    around the update launches only (the checks are outside it)."""

    def __init__(self, n, re, K, prec):
        import torch
        S = _S()
        self.n, self.K = n, K
        self.h = S.smrt_create(n, n, W.cavity_tau(n, U_LID, re), U_LID, W.CAVITY)
        S.smrt_set_option(self.h, S.SMRT_OPT_PRECISION, prec)
        S.smrt_set_option(self.h, S.SMRT_OPT_CHECK_DIVERGENCE, 0)
        self.t = 0
        self.step_ms = 0.0
        self.u_prev = _u_of(self.h, n)
        self._ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))

    def init(self, rho, u):
        S = _S()
        S.smrt_init_macros(self.h, rho, u)
        self.u_prev = _u_of(self.h, self.n)

    def advance(self):
        import torch
        S = _S()
        a, b = self._ev
        a.record()
        S.smrt_step(self.h, self.K)
        b.record()
        self.t += self.K
        u = _u_of(self.h, self.n)
        torch.cuda.synchronize()
        self.step_ms += a.elapsed_time(b)
        norm = float(u.norm())
        r = float((u - self.u_prev).norm()) / (self.K * norm) if norm > 0 else 0.0
        self.u_prev = u
        if not math.isfinite(r):
            raise FloatingPointError("cavity diverged at t = %d" % self.t)
        return u, r

    def close(self):
        _S().smrt_destroy(self.h)


def _converge(tr, tol, ref_tol, ref_factor, max_steps):
    """Advances a tracked cavity until its stride residual first falls below `tol` (steps_tol), then on
    until it falls below `ref_tol` or steps_tol x ref_factor: its own converged field.  Returns the
    velocity at every check (float32), steps_tol (None if capped), the final field, steps and residual."""
    snaps, steps_tol, r = [], None, 1.0
    while tr.t < max_steps:
        u, r = tr.advance()
        snaps.append(u.float())
        if steps_tol is None and r < tol:
            steps_tol = tr.t
        if steps_tol is not None and (r < ref_tol or tr.t >= ref_factor * steps_tol):
            break
    return snaps, steps_tol, tr.u_prev, tr.t, r


def time_to_same_error(net, res, n: int, prec: int = None, tol: float = 1e-7, ref_tol: float = 1e-11,
                       levels=(), check_every: int = 1000, max_steps: int = 400000, train_n: int = 256,
                       ref_factor: int = 6):
    """Time to steady state at the same error, cold start vs learned warm start, per Re (n x n cavity).

    Each run -- cold from rest, warm from f^eq of the network's prediction -- goes on past the plain
    method's steady criterion (stride residual < `tol`) until its residual falls below `ref_tol` (four
    decades lower) or its steps reach ref_factor times the criterion's: that is the run's own converged
    field u_inf, decided by the plain solver alone.  The error of a run at step t is
    e(t) = max over nodes |u(t) - u_inf| / U_lid.  The same error is the cold run's e at its criterion;
    the warm run's time to steady is its first check with e at most that (and, for each of `levels`,
    at most that level).  The two converged fields are compared as well (final_diff): the steady state
    of this update with halfway bounce-back is not unique -- on the FP64 oracle a 32^2 cavity started
    from a perturbed field settles 1e-3 U away from the cold start's, with its residual at rounding
    level -- and in FP32 each run also freezes at its own fixed point once every correction rounds
    away.  Wall times are steps x the measured per-update time of the lattice (CUDA events over the
    update launches); the warm time adds the prediction (network, resampling, smrt_init_macros).
    A run that does not reach `tol` within max_steps is reported as capped and left out.  The
    prediction path is run once before the first timed prediction (its first call initialises the
    library's inference state, ~0.5 s, as the solver's first launches are warmed before timing);
    warm steps are counted in whole checks, so a warm run that reaches the error within the first
    check_every updates counts check_every."""
    import torch
    S = _S()
    if prec is None:
        prec = S.SMRT_PREC_F32
    if net is not None and len(res):
        predict_fields(net, [res[0]], n, train_n)
        torch.cuda.synchronize()
    out = []
    for re in res:
        row = {"re": re, "n": n, "prec": {0: "f64", 1: "f32"}.get(prec, prec)}
        cold = _Tracked(n, re, check_every, prec)
        snaps_c, steps_cold, uinf_c, end_c, r_c = _converge(cold, tol, ref_tol, ref_factor, max_steps)
        ms_per_step = cold.step_ms / max(cold.t, 1)
        cold.close()
        if steps_cold is None:
            row.update(capped=True, cold_steps=end_c, cold_residual=r_c)
            out.append(row)
            continue
        ref_c = uinf_c.float()
        e_c = [float((x - ref_c).abs().amax()) / U_LID for x in snaps_c]
        del snaps_c
        e_cold = e_c[steps_cold // check_every - 1]

        warm = _Tracked(n, re, check_every, prec)
        torch.cuda.synchronize()
        tp = time.perf_counter()
        rho_p, u_p = predict_fields(net, [re], n, train_n)
        warm.init(rho_p[0], u_p[0])
        torch.cuda.synchronize()
        predict_s = time.perf_counter() - tp
        u_w0 = warm.u_prev.float()
        snaps_w, steps_tol_w, uinf_w, end_w, r_w = _converge(warm, tol, ref_tol, ref_factor, max_steps)
        warm.close()
        ref_w = uinf_w.float()
        e_w = [float((u_w0 - ref_w).abs().amax()) / U_LID] + \
              [float((x - ref_w).abs().amax()) / U_LID for x in snaps_w]
        del snaps_w
        row.update(capped=False, cold_steps=steps_cold, cold_end_steps=end_c, cold_end_residual=r_c,
                   cold_error=e_cold, warm_initial_error=e_w[0], warm_steps_tol=steps_tol_w,
                   warm_end_steps=end_w, warm_end_residual=r_w,
                   warm_error_at_tol=(e_w[steps_tol_w // check_every] if steps_tol_w else None),
                   final_diff=float((uinf_w - uinf_c).abs().amax()) / U_LID,
                   initial_diff=float((u_w0 - ref_c).abs().amax()) / U_LID,
                   ms_per_step=ms_per_step, predict_s=predict_s, targets={})
        for name, lv in [("same_error", e_cold)] + [("level_%g" % x, x) for x in levels]:
            kc = next((i for i, e in enumerate(e_c) if e <= lv), None)
            kw = next((i for i, e in enumerate(e_w) if e <= lv), None)
            c = None if kc is None else (kc + 1) * check_every
            w = None if kw is None else kw * check_every          # e_w[0] is the start, before any step
            t = {"error": lv, "cold_steps": c, "warm_steps": w}
            if c and w is not None:
                t["cold_s"] = c * ms_per_step * 1e-3
                t["warm_s"] = w * ms_per_step * 1e-3 + predict_s
                t["steps_factor"] = c / max(w, check_every)
                t["wall_factor"] = t["cold_s"] / t["warm_s"]
            row["targets"][name] = t
        out.append(row)
    return out
