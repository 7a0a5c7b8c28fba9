"""The learned warm start end to end at a small size: a dataset from the FP64
solver, training with the library's BF16 kernels, and the solves started from
the network's prediction against those started from the previous phi.

What the network gains is measured, not assumed: the test requires that
training lowers the loss, that the solves from the prediction reach the same
tolerance and the same discrete solution, that the prediction is closer to
the new solution than the previous phi, and that its solves take no more
V-cycles.  (The initial residual is not the criterion: the prediction's BF16
rounding noise is high-frequency, which the Laplacian amplifies and the first
smoothing sweep removes.)"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cmg():
    import __graft_entry__ as ge
    ge.build()
    from paper_2604_06035_gb300 import cmg as _c
    return _c


def test_warmstart_trains_and_helps(cmg):
    import torch
    from oracle import unet_oracle as U
    from paper_2604_06035_gb300 import warmstart as W
    ctx = cmg.cmg_ctx_create(0)
    try:
        data = W.build_dataset(ctx, n_traj=12, n_steps=8, D=32, seed=11)
        net = cmg.cmg_unet_create(ctx, 32, 4)
        p = U.init_params(12)
        p[-17:-1] = 0.0  # start from "delta = 0", i.e. from the previous phi
        cmg.cmg_unet_set_params(net, p.astype(np.float32))
        before, _ = W.evaluate(ctx, net, data, [10, 11])
        losses = W.train(net, data, list(range(10)), epochs=12, batch=4, lr=2e-3)
        after, rows = W.evaluate(ctx, net, data, [10, 11])
        assert losses[-1] < 0.7 * losses[0]
        assert after["rel_final_net"] <= 1e-10
        # the untrained network is exactly the previous phi
        assert abs(before["rel0_net"] - before["rel0_prev"]) <= 1e-6 * before["rel0_prev"]
        # the trained network is a better starting point than the previous phi
        assert abs(before["err_net"] - before["err_prev"]) <= 1e-6 * before["err_prev"]
        assert after["err_net"] < 0.7 * after["err_prev"]
        assert after["cycles_net"] <= after["cycles_prev"]
        # both starts converge to the same discrete solution
        S = W.PeriodicSolver(ctx, 32)
        rho, prev = data["rho"][10, 5], data["phi"][10, 4]
        a, _ = S.solve(rho, prev, 1e-12)
        pred = W.predict(S, net, rho, prev)
        b, _ = S.solve(rho, pred, 1e-12)
        assert float((a - b).abs().max() / a.abs().max()) <= 1e-9
        del net, S
        torch.cuda.synchronize()
    finally:
        cmg.cmg_ctx_destroy(ctx)
