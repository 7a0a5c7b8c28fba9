"""Learned warm start for the periodic level solve: the dataset comes from the
library's own FP64 solver, the U-Net is trained with the library's BF16
kernels (cmg_unet_*), and the gain is measured in V-cycles and device time to
a relative residual against plain multigrid started from the previous phi.

Workload (a stand-in for evolving cosmological densities): periodic D^3
blocks, ln rho_{t+1} = ln rho_t + eps g (inputs.warmstart_trajectory); phi_t
is solved to 1e-12 and each pair maps (rho_{t+1}, phi_t) to phi_{t+1}.  Whole
trajectories are held out for evaluation.

The network sees phi_t through its FP64 residual r = f_{t+1} - L phi_t for
the new density (the solver's own residual kernel), and predicts
phi_t + rms(r) delta.  The correction it has to learn, phi_{t+1} - phi_t, is
the zero-mean solution of L e = r: a fixed smooth linear map of r, which a
BF16 network can approximate, whereas L phi_t itself is lost when phi_t is
rounded to BF16 (the BF16 step is ~0.4% of |phi|, far above the change of
phi between steps).

Python here only orders the calls; every field stays on the device.
"""
import time

import numpy as np

from . import cmg, inputs


# (name, input channels, output channels) of the ten 3x3x3 convolutions in
# the order of the parameter vector (include/cmg.h), then the 16 + 1 head.
LAYERS = [("enc0a", 16, 16), ("enc0b", 16, 16), ("enc1a", 16, 32), ("enc1b", 32, 32), ("bota", 32, 64),
          ("botb", 64, 64), ("dec1a", 96, 32), ("dec1b", 32, 32), ("dec0a", 48, 16), ("dec0b", 16, 16)]


def init_params(seed, zero_head=True):
    """He-normal convolution weights, zero biases, the first layer's unused
    input channels 2..15 zero; the head zero when zero_head (the untrained
    network then returns its base, i.e. phi_prev).  FP32 vector."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, ci, co in LAYERS:
        w = rng.normal(0.0, np.sqrt(2.0 / (27 * ci)), size=(co, 27, ci))
        if name == "enc0a":
            w[:, :, 2:] = 0.0
        parts += [w.ravel(), np.zeros(co)]
    head = np.zeros(16) if zero_head else rng.normal(0.0, 0.05, size=16)
    parts += [head, np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


class PeriodicSolver:
    """A full periodic level of D^3 cells, with dense [D, D, D] (z, y, x)
    device fields in and out (converted to octs by cmg_dense_octs)."""

    def __init__(self, ctx, D):
        import torch
        self.ctx, self.D = ctx, D
        lev = int(round(np.log2(D)))
        coords = torch.from_numpy(inputs.uniform_oct_coords(lev)).cuda()
        self.level = cmg.cmg_level_build(ctx, lev, cmg.cmg_morton_encode(ctx, coords))
        self.octs = torch.empty(((D // 2) ** 3, 8), dtype=torch.float64, device="cuda")
        self.dense = torch.empty((D, D, D), dtype=torch.float64, device="cuda")

    def _load(self, rho, phi0):
        r = rho.to(dtype=self.dense.dtype).contiguous()
        cmg.cmg_dense_octs(self.ctx, r, self.D, self.octs, 1)
        cmg.cmg_level_set_density(self.level, self.octs, float(r.mean().item()))
        if phi0 is None:
            self.octs.zero_()
        else:
            cmg.cmg_dense_octs(self.ctx, phi0.to(dtype=self.dense.dtype).contiguous(), self.D, self.octs, 1)
        cmg.cmg_level_set_phi(self.level, self.octs)

    def _dense_out(self):
        out = self.dense.new_empty(self.dense.shape)
        cmg.cmg_dense_octs(self.ctx, self.octs, self.D, out, 0)
        return out

    def residual(self, rho, phi):
        """r = f - L phi (FP64, dense device tensor) for density rho."""
        self._load(rho, phi)
        cmg.cmg_level_get_residual(self.level, device=True, out=self.octs)
        return self._dense_out()

    def solve(self, rho, phi0=None, tol=1e-10, precision=cmg.CMG_PREC_FP64):
        """rho, phi0: dense device tensors (any float dtype).  Returns (phi as a
        dense float64 device tensor, solve statistics)."""
        self._load(rho, phi0)
        rc, st = cmg.cmg_level_solve(self.level, tol=tol, precision=precision)
        cmg.cmg_level_get_phi(self.level, device=True, out=self.octs)
        return self._dense_out(), st


def build_dataset(ctx, n_traj, n_steps, D=64, seed=5, eps=0.05, sigma=1.5, tol=1e-12):
    """Densities, solved potentials ([n_traj, n_steps + 1, D, D, D]) and the
    residuals of phi_t for rho_{t+1} ([n_traj, n_steps, D, D, D]), float32
    device tensors."""
    import torch
    S = PeriodicSolver(ctx, D)
    rho = torch.empty((n_traj, n_steps + 1, D, D, D), dtype=torch.float32, device="cuda")
    phi = torch.empty_like(rho)
    res = torch.empty((n_traj, n_steps, D, D, D), dtype=torch.float32, device="cuda")
    t0 = time.perf_counter()
    solves = 0
    for k in range(n_traj):
        traj = torch.from_numpy(inputs.warmstart_trajectory(D, n_steps, sigma, eps, seed, k)).cuda()
        prev = None
        for t in range(n_steps + 1):
            if prev is not None:
                res[k, t - 1] = S.residual(traj[t], prev).float()
            p, st = S.solve(traj[t], prev, tol)
            prev = p
            rho[k, t] = traj[t].float()
            phi[k, t] = p.float()
            solves += 1
    torch.cuda.synchronize()
    return {"rho": rho, "phi": phi, "res": res, "D": D, "n_traj": n_traj, "n_steps": n_steps,
            "seconds": time.perf_counter() - t0, "solves": solves}


def _pairs(data, trajs):
    return [(k, t) for k in trajs for t in range(data["n_steps"])]


def _batch(data, pairs):
    """(rho_{t+1}, r_t, phi_t, phi_{t+1}) stacked over the pairs."""
    import torch
    k = torch.tensor([p[0] for p in pairs], device="cuda")
    t = torch.tensor([p[1] for p in pairs], device="cuda")
    return (data["rho"][k, t + 1].contiguous(), data["res"][k, t].contiguous(),
            data["phi"][k, t].contiguous(), data["phi"][k, t + 1].contiguous())


def output_scale(data, trajs):
    """The rms over the pairs of (phi_{t+1} - phi_t) / rms(r_t): the network's
    output scale, so that the delta it regresses is O(1)."""
    import torch
    acc = 0.0
    pairs = _pairs(data, trajs)
    for k, t in pairs:
        r = data["res"][k, t].double()
        d = (data["phi"][k, t + 1] - data["phi"][k, t]).double()
        acc += float((d.pow(2).mean() / r.pow(2).mean()).item())
    return float(np.sqrt(acc / len(pairs)))


def train(net, data, train_trajs, epochs=10, batch=4, lr=1e-3, seconds=None, seed=0, calibrate=True,
          warmup_steps=200, clip=4.0):
    """Adam on the mean squared error of delta with a cosine learning-rate
    decay over `epochs`, or over a wall-clock budget of `seconds` when given
    (then as many epochs as fit), after a linear warm-up over the first
    `warmup_steps` steps (full-size first steps could switch off whole ReLU
    layers of the freshly initialised network, leaving it at a zero
    prediction); each step's gradient norm is capped at `clip` times its
    running mean (0: no cap), since a single outsized step has left the
    network at a zero prediction too; the output scale is set from the
    training pairs first when calibrate.  Returns the per-epoch mean loss."""
    rng = np.random.default_rng(seed)
    pairs = _pairs(data, train_trajs)
    if calibrate:
        cmg.cmg_unet_set_output_scale(net, output_scale(data, train_trajs))
    cmg.cmg_unet_set_grad_clip(net, clip)
    losses = []
    t0 = time.perf_counter()
    steps_total = epochs * ((len(pairs) + batch - 1) // batch)
    if seconds is None:
        warmup_steps = min(warmup_steps, steps_total // 10)
    step = 0
    ep = 0
    while True:
        if seconds is None and ep >= epochs:
            break
        order = rng.permutation(len(pairs))
        acc, nb = 0.0, 0
        for i in range(0, len(pairs), batch):
            if seconds is not None:
                progress = min(1.0, (time.perf_counter() - t0) / seconds)
            else:
                progress = step / steps_total
            chunk = [pairs[j] for j in order[i:i + batch]]
            rho, r, prev, nxt = _batch(data, chunk)
            loss, _ = cmg.cmg_unet_gradients(net, rho, r, nxt, base=prev, grads=False)
            warm = min(1.0, (step + 1) / warmup_steps) if warmup_steps > 0 else 1.0
            cmg.cmg_unet_adam_step(net, lr * warm * 0.5 * (1 + np.cos(np.pi * progress)))
            step += 1
            acc += loss / len(chunk)
            nb += 1
            if seconds is not None and progress >= 1.0:
                break
        losses.append(float((acc / (nb * data["D"] ** 3)).item()))
        ep += 1
        if seconds is not None and time.perf_counter() - t0 >= seconds:
            break
    return losses


def predict(S, net, rho, prev):
    """The warm start for density rho from the previous potential prev (dense
    device tensors): residual of prev, then the network."""
    r = S.residual(rho, prev).float()
    pred = cmg.cmg_unet_forward(net, rho[None].float().contiguous(), r[None].contiguous(),
                                base=prev[None].float().contiguous())
    return pred[0]


def _rel_err(a, ref):
    """Relative L2 error of a against ref, constants removed (they are the
    periodic operator's null space)."""
    d = (a - a.mean()) - (ref - ref.mean())
    return float((d.norm() / (ref - ref.mean()).norm()).item())


def evaluate(ctx, net, data, test_trajs, tol=1e-10, precision=cmg.CMG_PREC_FP64):
    """Per held-out pair: V-cycles, device ms and initial relative residual of
    the solve started from phi_t and from the network's prediction (and from
    zero), and the error of both starts against phi_{t+1}; the warm start's
    own cost (residual + network) is timed with CUDA events."""
    import torch
    S = PeriodicSolver(ctx, data["D"])
    rows = []
    for k, t in _pairs(data, test_trajs):
        rho = data["rho"][k, t + 1]
        prev = data["phi"][k, t]
        _, st_prev = S.solve(rho, prev, tol, precision)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        pred = predict(S, net, rho, prev)
        e1.record()
        torch.cuda.synchronize()
        nxt = data["phi"][k, t + 1].double()
        err_prev, err_net = _rel_err(prev.double(), nxt), _rel_err(pred.double(), nxt)
        _, st_net = S.solve(rho, pred, tol, precision)
        _, st_zero = S.solve(rho, None, tol, precision)
        rows.append({"cycles_prev": st_prev["cycles"], "cycles_net": st_net["cycles"],
                     "cycles_zero": st_zero["cycles"], "ms_prev": st_prev["ms"], "ms_net": st_net["ms"],
                     "ms_zero": st_zero["ms"], "ms_infer": e0.elapsed_time(e1),
                     "rel0_prev": st_prev["rel_initial"], "rel0_net": st_net["rel_initial"],
                     "rel_final_net": st_net["rel_final"], "err_prev": err_prev, "err_net": err_net})
    keys = rows[0].keys()
    mean = {k: float(np.mean([r[k] for r in rows])) for k in keys}
    mean["pairs"] = len(rows)
    return mean, rows
