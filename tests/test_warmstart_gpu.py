"""Learned warm start end to end on a small scale: solver-generated data, U-Net
training with libsmrt's kernels, and a warm start that reaches the same steady
state as the cold start in fewer steps."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_warm_start_reaches_the_same_steady_state_faster():
    import torch
    from paper_2409_01076_gb300 import warmstart as WS
    from paper_2409_01076_gb300.unet import UNet
    torch.cuda.set_device(0)
    n = 32
    res = WS.sample_res(24, seed=5, lo=100.0, hi=1000.0)
    targets, info = WS.generate_dataset(res, n, tol=1e-7, check_every=200, max_steps=200000)
    assert info["converged"] == len(res), info
    net = UNet(base=8, seed=2)
    hist, _ = WS.train(net, res, targets, iters=2000, batch=8, lr=3e-3, log_every=250)
    assert hist[-1][1] < 0.01 * hist[0][1], hist
    held = [180.0, 600.0]
    cold, fc = WS.time_to_steady(held, n, None, 1e-7, 200, 200000, train_n=n)
    warm, fw = WS.time_to_steady(held, n, net, 1e-7, 200, 200000, train_n=n)
    assert cold["state"] == [1, 1] and warm["state"] == [1, 1], (cold, warm)
    _, u_pred = WS.predict_fields(net, held, n, train_n=n)
    for k in range(2):
        err = float((u_pred[k] - fc[k]).norm() / fc[k].norm())
        assert err < 0.1, (k, err, hist)                     # held-out Re: the guess is close
        assert warm["steps"][k] < cold["steps"][k], (cold["steps"], warm["steps"], err)
        # both runs end at the solver's own steady state, not the network's guess
        assert float((fc[k] - fw[k]).abs().max()) / WS.U_LID < 1e-3
