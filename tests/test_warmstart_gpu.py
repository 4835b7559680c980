"""Learned warm start end to end on a small scale: solver-generated data, U-Net
training with libsmrt's kernels, and a warm start that reaches the same steady
state as the cold start in fewer steps."""
import numpy as np
import pytest

import paper_2409_01076_gb300 as S

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
    # time to steady at the same error: each run's distance to its own converged field, the warm run
    # against the error the plain method has at its own criterion
    rows = WS.time_to_same_error(net, held, n, S.SMRT_PREC_F64, 1e-7, 1e-11, (1e-3,), 200, 400000, train_n=n)
    for row in rows:
        assert not row["capped"], row
        assert row["cold_end_steps"] >= row["cold_steps"] and row["cold_end_residual"] < 1e-9, row
        assert 0.0 < row["cold_error"] < 1e-3, row
        assert row["warm_initial_error"] > row["cold_error"], row       # the guess alone is not enough
        t = row["targets"]["same_error"]
        assert t["cold_steps"] is not None and t["warm_steps"] is not None, row
        assert t["warm_steps"] < t["cold_steps"], row
        assert t["steps_factor"] > 1.0 and t["wall_factor"] > 1.0, row
        assert row["targets"]["level_0.001"]["warm_steps"] is not None, row
        assert row["final_diff"] < 1e-2, row
