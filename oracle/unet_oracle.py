"""Plain FP64 reference of the warm-start U-Net.  TEST INFRASTRUCTURE ONLY.

The network (not in the paper; it is the learned initial guess of the
benchmark's fifth workload): a 3-level 3-D U-Net with 16/32/64 channels on a
periodic D^3 block, inputs (rho, phi_prev), output the change of phi.

  enc0a 16->16, enc0b 16->16                 at D      (skip s0)
  avg-pool 2
  enc1a 16->32, enc1b 32->32                 at D/2    (skip s1)
  avg-pool 2
  bota 32->64, botb 64->64                   at D/4
  nearest x2, concat [up, s1] (64+32)
  dec1a 96->32, dec1b 32->32                 at D/2
  nearest x2, concat [up, s0] (32+16)
  dec0a 48->16, dec0b 16->16                 at D
  head 1x1x1 16->1 (linear): delta

Every 3x3x3 convolution has circular padding, a bias and a ReLU.  Input
channels: 0 = (rho - mean rho) / std rho, 1 = field / rms field, 2..15 zero.
The prediction is base + c rms(field) delta (base defaults to field, c is the
output scale).

Activations are channels-last arrays [D, D, D, C] indexed [z, y, x, c]; conv
weights are [Cout, 27, Cin] with tap t = 9 (dz+1) + 3 (dy+1) + (dx+1); the
flat parameter vector lists, layer by layer, the weights then the biases,
then the head's 16 weights and bias.

bf16=True reproduces where the GPU network rounds to bfloat16 (round to
nearest even): the conv weights, every stored activation (conv outputs after
bias and ReLU, pooled maps) and every stored gradient that feeds a
convolution; all arithmetic is FP64 in between.
"""
import numpy as np

LAYERS = [("enc0a", 16, 16, 0), ("enc0b", 16, 16, 0), ("enc1a", 16, 32, 1), ("enc1b", 32, 32, 1),
          ("bota", 32, 64, 2), ("botb", 64, 64, 2), ("dec1a", 96, 32, 1), ("dec1b", 32, 32, 1),
          ("dec0a", 48, 16, 0), ("dec0b", 16, 16, 0)]
TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def n_params():
    return sum(co * 27 * ci + co for _, ci, co, _ in LAYERS) + 17


def unpack(params):
    p = np.asarray(params, dtype=np.float64)
    out, o = {}, 0
    for name, ci, co, _ in LAYERS:
        w = p[o:o + co * 27 * ci].reshape(co, 27, ci)
        o += co * 27 * ci
        b = p[o:o + co]
        o += co
        out[name] = (w, b)
    out["head"] = (p[o:o + 16], p[o + 16])
    return out


def init_params(seed):
    """He-normal weights (zero biases), the channels 2..15 of the first layer zero."""
    rng = np.random.default_rng(seed)
    parts = []
    for name, ci, co, _ in LAYERS:
        w = rng.normal(0.0, np.sqrt(2.0 / (27 * ci)), size=(co, 27, ci))
        if name == "enc0a":
            w[:, :, 2:] = 0.0
        parts += [w.ravel(), np.zeros(co)]
    parts += [rng.normal(0.0, 0.05, size=16), np.zeros(1)]
    return np.concatenate(parts)


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a32 = np.asarray(a, dtype=np.float32)
    bits = a32.view(np.uint32).astype(np.uint64)
    bits = (bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)


def shift(x, d):
    """y[z, y, x] = x[z + dz, y + dy, x + dx] (periodic)."""
    return np.roll(x, (-d[0], -d[1], -d[2]), axis=(0, 1, 2))


def conv(x, w, b):
    out = np.broadcast_to(b, x.shape[:3] + (w.shape[0],)).copy()
    for t, d in enumerate(TAPS):
        out += shift(x, d) @ w[:, t, :].T
    return out


def conv_bwd(x, w, dout):
    dw = np.zeros_like(w)
    dx = np.zeros_like(x)
    V = np.prod(x.shape[:3])
    for t, d in enumerate(TAPS):
        xs = shift(x, d)
        dw[:, t, :] = dout.reshape(V, -1).T @ xs.reshape(V, -1)
        dx += np.roll(dout @ w[:, t, :], d, axis=(0, 1, 2))
    return dx, dw, dout.sum(axis=(0, 1, 2))


def pool(x):
    D = x.shape[0] // 2
    return x.reshape(D, 2, D, 2, D, 2, -1).mean(axis=(1, 3, 5))


def pool_bwd(d):
    return np.repeat(np.repeat(np.repeat(d, 2, 0), 2, 1), 2, 2) / 8.0


def up(x):
    return np.repeat(np.repeat(np.repeat(x, 2, 0), 2, 1), 2, 2)


def up_bwd(d):
    D = d.shape[0] // 2
    return d.reshape(D, 2, D, 2, D, 2, -1).sum(axis=(1, 3, 5))


def inputs(rho, field):
    """Network input [D,D,D,16] and the output scale (rms of field)."""
    s = np.sqrt(np.mean(field ** 2))
    x = np.zeros(rho.shape + (16,))
    x[..., 0] = (rho - rho.mean()) / rho.std()
    x[..., 1] = field / s
    return x, s


def forward(params, rho, field, base=None, bf=False, scale=1.0):
    """Returns (delta [D,D,D], base + scale rms(field) delta, cache); base
    defaults to field."""
    P = unpack(params)
    R = bf16 if bf else (lambda a: a)
    if base is None:
        base = field
    x, s = inputs(rho, field)
    s = s * scale
    x = R(x)
    cache = {"x": x, "s": s}

    def layer(name, a):
        w, b = P[name]
        out = R(np.maximum(conv(a, R(w), b), 0.0))
        cache[name] = (a, out)
        return out

    s0 = layer("enc0b", layer("enc0a", x))
    s1 = layer("enc1b", layer("enc1a", R(pool(s0))))
    bt = layer("botb", layer("bota", R(pool(s1))))
    d1 = layer("dec1b", layer("dec1a", np.concatenate([up(bt), s1], axis=-1)))
    d0 = layer("dec0b", layer("dec0a", np.concatenate([up(d1), s0], axis=-1)))
    hw, hb = P["head"]
    delta = d0 @ hw + hb
    cache["d0"] = d0
    return delta, base + s * delta, cache


def loss_and_grads(params, rho, field, target, base=None, bf=False, scale=1.0):
    """MSE between delta and (target - base) / (scale rms(field)) over the
    voxels (base defaults to field); returns (loss, flat gradient)."""
    P = unpack(params)
    R = bf16 if bf else (lambda a: a)
    if base is None:
        base = field
    delta, _, c = forward(params, rho, field, base, bf, scale)
    target = (target - base) / c["s"]
    V = delta.size
    loss = np.mean((delta - target) ** 2)
    g = {}
    dd = 2.0 * (delta - target) / V
    hw, hb = P["head"]
    g["head"] = ((c["d0"] * dd[..., None]).sum(axis=(0, 1, 2)), dd.sum())
    dact = R(dd[..., None] * hw)

    def back(name, dact):
        a, out = c[name]
        w, b = P[name]
        dpre = R(dact * (out > 0))
        dx, dw, db = conv_bwd(a, R(w), dpre)
        g[name] = (dw, db)
        return R(dx)

    dx = back("dec0a", back("dec0b", dact))
    d_up0, d_s0 = R(dx[..., :32]), dx[..., 32:]
    dx = back("dec1a", back("dec1b", R(up_bwd(d_up0))))
    d_up1, d_s1 = R(dx[..., :64]), dx[..., 64:]
    dx = back("bota", back("botb", R(up_bwd(d_up1))))
    d_s1 = R(d_s1 + pool_bwd(dx))
    dx = back("enc1a", back("enc1b", d_s1))
    d_s0 = R(d_s0 + pool_bwd(dx))
    back("enc0a", back("enc0b", d_s0))
    parts = []
    for name, ci, co, _ in LAYERS:
        parts += [g[name][0].ravel(), g[name][1]]
    parts += [g["head"][0], np.array([g["head"][1]])]
    return loss, np.concatenate(parts)
