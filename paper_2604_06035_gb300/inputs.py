"""Seeded synthetic inputs for the oct-grid Poisson solve.

This module holds no arithmetic of the method (no Morton keys, no hashing, no
Poisson operator): it produces integer oct coordinates and densities in
oct-major layout, which both the CUDA library and the CPU oracle consume.

Stand-ins for the paper's Cosmo256/512/1024 MUSIC initial conditions (Sec. 7.1),
which are not available: Gaussian random fields with P(k) ~ k^-2, lognormal
densities, overdensity-flagged refinement (threshold 8 rho_bar, one-cell
dilation) and mass-conserving child densities.

Layout conventions (shared by both sides of every parity test):
  * level l has 2^l cells and 2^(l-1) octs per axis (n_x = 1, box [0,1)^3);
  * a dense cell array is indexed field[x, y, z];
  * an oct-major array is [n_octs, 8] with child c = bx + 2 by + 4 bz;
  * uniform levels list their octs in lexicographic order, x fastest.
"""
import numpy as np


# ----------------------------------------------------------------- layouts

def uniform_oct_coords(level):
    """All oct coordinates of a full level, x fastest: uint32 [n^3, 3]."""
    n = 1 << (level - 1)
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1).astype(np.uint32)


def child_offsets():
    """(bx, by, bz) of child c = bx + 2 by + 4 bz, as int [8, 3]."""
    c = np.arange(8)
    return np.stack([c & 1, (c >> 1) & 1, (c >> 2) & 1], axis=1)


def dense_to_octs(field, coords):
    """Gather a dense cell array field[x, y, z] into oct-major [n, 8]."""
    off = child_offsets()
    X = 2 * coords[:, None, :].astype(np.int64) + off[None, :, :]
    return np.ascontiguousarray(field[X[..., 0], X[..., 1], X[..., 2]])


def octs_to_dense(values, coords, n_cells):
    """Scatter oct-major [n, 8] back into a dense array (unset cells = NaN)."""
    out = np.full((n_cells,) * 3, np.nan, dtype=values.dtype)
    off = child_offsets()
    X = 2 * coords[:, None, :].astype(np.int64) + off[None, :, :]
    out[X[..., 0], X[..., 1], X[..., 2]] = values
    return out


# --------------------------------------------------------------- densities

def grf(n, rms, seed, slope=-2.0):
    """Periodic Gaussian random field on n^3 cells, P(k) ~ |k|^slope for integer
    0 < |k| <= n/2 (DC and modes beyond Nyquist zeroed), rescaled to rms."""
    rng = np.random.default_rng(seed)
    white = rng.standard_normal((n, n, n))
    wk = np.fft.rfftn(white)
    kx = np.fft.fftfreq(n) * n
    kz = np.fft.rfftfreq(n) * n
    k = np.sqrt(kx[:, None, None] ** 2 + kx[None, :, None] ** 2 + kz[None, None, :] ** 2)
    amp = np.zeros_like(k)
    sel = (k > 0) & (k <= n / 2)
    amp[sel] = k[sel] ** (slope / 2.0)
    g = np.fft.irfftn(wk * amp, s=(n, n, n), axes=(0, 1, 2))
    g -= g.mean()
    return g * (rms / np.sqrt(np.mean(g * g)))


def lognormal(n, sigma, seed):
    """rho = exp(sigma g) / mean(exp(sigma g)), g a unit-rms k^-2 GRF: mean 1,
    sigma_ln(rho) = sigma exactly."""
    g = grf(n, 1.0, seed)
    e = np.exp(sigma * g)
    return e / e.mean()


# -------------------------------------------------------------- refinement

def _cell_index(cells, size):
    """Sorted linear keys of a level's cells (periodic box of size^3 cells) and a
    lookup q [k, 3] -> position in `cells` or -1."""
    lin = lambda c: ((c[:, 0] % size) * size + (c[:, 1] % size)) * size + (c[:, 2] % size)
    keys = lin(cells)
    order = np.argsort(keys, kind="stable")
    sk = keys[order]

    def find(q):
        k = lin(q)
        pos = np.minimum(np.searchsorted(sk, k), len(sk) - 1)
        return np.where(sk[pos] == k, order[pos], -1)
    return find


def refine_cells(level, coords, rho_octs, threshold):
    """Cells of a level to refine: rho > threshold, dilated by one cell over the
    6 face neighbours among existing cells (periodic), keeping only cells whose
    26 neighbours all exist (so that the new octs' coarse-fine ghost stencils
    exist).  A 26-neighbour dilation of the k^-2 lognormal flags refines ~23 %
    of the volume at sigma = 1.5; the face dilation gives ~9 %, inside the
    5-10 % band the two-level workload is specified with.

    coords: oct coords [n, 3] of the level, rho_octs [n, 8].  Returns the global
    cell coordinates [m, 3] (uint32) in oct-major order of the level, i.e. the
    oct coordinates of the new octs one level down, and their positions in the
    level's flattened [n * 8] cell order.  Sparse: lookups in the sorted cell
    keys, so that deep levels need no dense volume."""
    off = child_offsets()
    cells = (2 * coords[:, None, :].astype(np.int64) + off[None, :, :]).reshape(-1, 3)
    size = 1 << level
    find = _cell_index(cells, size)
    flag = rho_octs.reshape(-1) > threshold
    fl = flag.copy()
    fc = cells[flag]
    for axis in range(3):
        for s in (-1, 1):
            q = fc.copy()
            q[:, axis] += s
            j = find(q)
            fl[j[j >= 0]] = True
    cand = np.nonzero(fl)[0]
    cc = cells[cand]
    # a cell exists iff its oct does: a dense oct-occupancy grid ((size/2)^3
    # bytes) answers the 26 neighbour tests
    half = size >> 1
    occ = np.zeros(half ** 3, dtype=bool)
    co = coords.astype(np.int64)
    occ[(co[:, 0] * half + co[:, 1]) * half + co[:, 2]] = True
    # oct coordinate of the neighbour cell along each axis for offsets -1, 0, 1
    ax = [[((cc[:, a] + d) & (size - 1)) >> 1 for d in (-1, 0, 1)] for a in range(3)]
    ok = np.ones(len(cand), dtype=bool)
    for i in range(3):
        for j in range(3):
            xy = (ax[0][i] * half + ax[1][j]) * half
            for k in range(3):
                if (i, j, k) != (1, 1, 1):
                    ok &= occ[xy + ax[2][k]]
    idx = cand[ok]
    return cells[idx].astype(np.uint32), idx


def child_density(rho_parent_cells, seed, level, sigma_inc=0.5):
    """Mass-conserving child densities: rho_child = rho_parent * e^{s xi} /
    mean_8(e^{s xi}), xi ~ N(0, 1) drawn per child.  Returns [m, 8]."""
    rng = np.random.default_rng([seed, level])
    xi = rng.standard_normal((len(rho_parent_cells), 8))
    e = np.exp(sigma_inc * xi)
    return rho_parent_cells[:, None] * e / e.mean(axis=1, keepdims=True)


# ------------------------------------------------------------------ configs

def periodic_grf_level(level, rms=0.5, seed=1):
    """Uniform periodic level with rho = 1 + delta, delta a k^-2 GRF of the
    given rms (the 32^3 plain-FP64 workload at level 5)."""
    n = 1 << level
    rho = 1.0 + grf(n, rms, seed)
    coords = uniform_oct_coords(level)
    return {"levels": [level], "coords": [coords], "rho": [dense_to_octs(rho, coords)], "rho_bar": 1.0}


def amr_lognormal(base_level, n_refine, sigma, seed, threshold=8.0, sigma_inc=0.5):
    """Periodic lognormal base level plus n_refine refined levels, each refining
    the cells above threshold * rho_bar (dilated, properly nested)."""
    n = 1 << base_level
    rho = lognormal(n, sigma, seed)
    coords = uniform_oct_coords(base_level)
    levels = [base_level]
    all_coords = [coords]
    all_rho = [dense_to_octs(rho, coords)]
    rho_bar = 1.0
    for r in range(n_refine):
        lev = base_level + r
        cells, idx = refine_cells(lev, all_coords[-1], all_rho[-1], threshold * rho_bar)
        if len(cells) == 0:
            break
        parent_rho = all_rho[-1].reshape(-1)[idx]  # density of each refined (parent) cell
        levels.append(lev + 1)
        all_coords.append(cells)
        all_rho.append(child_density(parent_rho, seed, lev + 1, sigma_inc))
    return {"levels": levels, "coords": all_coords, "rho": all_rho, "rho_bar": rho_bar}


def two_level_amr(base_level=7, sigma=1.5, seed=2):
    """Periodic lognormal base (sigma_ln rho = 1.5, k^-2) plus one level refined
    where rho > 8 rho_bar (the 128^3 two-level AMR workload at base level 7)."""
    return amr_lognormal(base_level, 1, sigma, seed)


def batched_patches(n_patches=512, n_min=64, n_max=200000, seed=4, level=11, sigma=1.5):
    """Independent refined patches for the batched solve.

    Patch sizes are log-uniform in [n_min, n_max] octs.  Patch k lives in its
    own cube of 128 octs per side (an 8 x 8 x 8 arrangement at `level`, whose
    box is 1024 octs wide) and is the compact, irregular set of the n_k octs
    of the central 64^3 sub-cube nearest to the sub-cube centre (distances
    perturbed by a seeded jitter), so patches are separated by at least 64
    octs and their multigrid hierarchies never touch.  Each patch has its own
    lognormal density (sigma_ln rho = sigma, k^-2 GRF on the 64^3 sub-cube;
    the patches draw from 16 seeded fields, each patch with its own seeded
    periodic shift and sign).  The parent level (level - 1) holds the parents
    of every patch oct dilated by one oct, with phi = a seeded sum of 8 low-k
    (|k| <= 4) sine modes at the parent cell centres (the smooth coarse field
    of the Dirichlet values).

    Returns dict(level, coords [N,3] uint32 (patches contiguous), offsets
    [n_patches+1], rho [N,8], parent_coords, parent_phi [M,8])."""
    if n_patches > 512:
        raise ValueError("at most 512 patches fit the 8^3 cube arrangement")
    rng = np.random.default_rng(seed)
    sizes = np.rint(np.exp(rng.uniform(np.log(n_min), np.log(n_max), n_patches))).astype(np.int64)
    sizes = np.clip(sizes, n_min, min(n_max, 64 ** 3))
    r = np.arange(64)
    z, y, x = np.meshgrid(r, r, r, indexing="ij")
    sub = np.stack([x.ravel(), y.ravel(), z.ravel()], 1)
    d2 = ((sub - 31.5) ** 2).sum(axis=1)
    n_shapes = 8
    orders = [np.argsort(d2 + np.random.default_rng([seed, s, 2]).uniform(0.0, 40.0, len(d2)), kind="stable")
              for s in range(n_shapes)]
    fields = []
    for s in range(16):
        e = np.exp(sigma * grf(64, 1.0, [seed, s, 1]))
        fields.append(e / e.mean())
    coords, rho, offsets, parents = [], [], [0], []
    for k in range(n_patches):
        prng = np.random.default_rng([seed, k])
        cells = sub[orders[k % n_shapes][:sizes[k]]]
        cube = np.array([k % 8, (k // 8) % 8, k // 64]) * 128 + 32
        coords.append((cells + cube).astype(np.uint32))
        shift = prng.integers(0, 64, size=3)
        sign = 1.0 if prng.uniform() < 0.5 else -1.0
        e = np.roll(fields[k % 16], tuple(shift), axis=(0, 1, 2))
        if sign < 0:
            e = 1.0 / e
            e /= e.mean()
        rho.append(child_density(e[cells[:, 0], cells[:, 1], cells[:, 2]], seed * 1000 + k, level, 0.5))
        offsets.append(offsets[-1] + sizes[k])
        # parent octs of the patch (a 32^3 window of level - 1), dilated by one oct
        m = np.zeros((34, 34, 34), dtype=bool)
        pc = cells >> 1
        m[pc[:, 0] + 1, pc[:, 1] + 1, pc[:, 2] + 1] = True
        d = m.copy()
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    d |= np.roll(m, (dx, dy, dz), axis=(0, 1, 2))
        parents.append(np.argwhere(d) - 1 + cube // 2)
    coords = np.concatenate(coords)
    rho = np.concatenate(rho)
    parent = np.ascontiguousarray(np.concatenate(parents), dtype=np.uint32)
    off = child_offsets()
    hp = 1.0 / (1 << (level - 1))
    X = (2 * parent[:, None, :].astype(np.float64) + off[None] + 0.5) * hp
    phi = np.zeros(X.shape[:2])
    for _ in range(8):
        kv = rng.integers(-4, 5, size=3)
        while not kv.any() or np.sqrt((kv ** 2).sum()) > 4:
            kv = rng.integers(-4, 5, size=3)
        amp, ph = rng.normal(0.0, 1.0), rng.uniform(0, 2 * np.pi)
        phi += amp * np.sin(2 * np.pi * (X @ kv) + ph)
    return {"level": level, "coords": coords, "offsets": np.array(offsets, dtype=np.int64), "rho": rho,
            "parent_coords": parent, "parent_phi": phi, "sizes": sizes}


def warmstart_trajectory(D=64, n_steps=20, sigma=1.5, eps=0.05, seed=5, traj=0):
    """Densities of one evolving periodic block for the learned warm start:
    ln rho_0 = sigma g_0, ln rho_{t+1} = ln rho_t + eps g_{t+1} (g unit-rms
    k^-2 GRFs seeded by (seed, traj, t)), each rho renormalised to mean 1.
    Returns float64 [n_steps + 1, D, D, D] indexed [t, z, y, x]."""
    out = np.empty((n_steps + 1, D, D, D))
    lnr = sigma * grf(D, 1.0, [seed, traj, 0])
    for t in range(n_steps + 1):
        if t:
            lnr = lnr + eps * grf(D, 1.0, [seed, traj, t])
        e = np.exp(lnr)
        out[t] = (e / e.mean()).transpose(2, 1, 0)
    return out


def mixed_amr(base_level=8, n_refine=3, sigma=2.0, seed=3):
    """Periodic lognormal base (sigma_ln rho = 2) plus three refined levels at
    threshold 8 rho_bar each (the 256^3 mixed-precision workload)."""
    return amr_lognormal(base_level, n_refine, sigma, seed)


def deep_zoom(base_level=4, top_level=30, cube=8, centre=(0.3217, 0.5791, 0.7123), seed=6):
    """A periodic base level plus a chain of refined levels up to top_level,
    each a cube of `cube`^3 octs centred on the same point (so every level sits
    inside its parent with the one-cell margin the coarse-fine stencils need).
    Levels above 22 need 128-bit Morton keys.  Densities: rho = 1 + a seeded
    uniform perturbation of amplitude 0.5 per cell.

    Returns {"levels", "coords": [n, 3] uint64 oct coordinates per level,
    "rho": [n, 8] per level, "rho_bar": base mean}."""
    rng = np.random.default_rng(seed)
    levels, coords, rhos = [base_level], [uniform_oct_coords(base_level).astype(np.uint64)], []
    for lev in range(base_level + 1, top_level + 1):
        npd = 1 << (lev - 1)
        assert cube + 4 <= npd, "the cube must leave room for its Dirichlet boundary"
        lo = [int(c * npd) - cube // 2 for c in centre]
        r = [np.arange(l, l + cube, dtype=np.uint64) for l in lo]
        z, y, x = np.meshgrid(r[2], r[1], r[0], indexing="ij")
        levels.append(lev)
        coords.append(np.stack([x.ravel(), y.ravel(), z.ravel()], 1))
    for c in coords:
        rhos.append(1.0 + 0.5 * (2.0 * rng.random((len(c), 8)) - 1.0))
    rho_bar = float(rhos[0].mean())
    return {"levels": levels, "coords": coords, "rho": rhos, "rho_bar": rho_bar}

