"""The seeded synthetic inputs have the structure their recipes state."""
import numpy as np

from paper_2604_06035_gb300 import inputs


def test_lognormal_statistics():
    rho = inputs.lognormal(32, 1.5, 2)
    assert abs(rho.mean() - 1.0) < 1e-12
    assert abs(np.log(rho).std() - 1.5) < 1e-12


def test_grf_spectrum_and_rms():
    g = inputs.grf(32, 0.5, 1)
    assert abs(np.sqrt(np.mean(g * g)) - 0.5) < 1e-12 and abs(g.mean()) < 1e-12
    p = np.abs(np.fft.fftn(g)) ** 2
    k = np.sqrt(sum(np.meshgrid(*[np.fft.fftfreq(32) * 32] * 3, indexing="ij")[i] ** 2 for i in range(3)))
    lo, hi = p[(k > 2) & (k < 3)].mean(), p[(k > 8) & (k < 9)].mean()
    assert 0.5 < (lo / hi) / (8.5 / 2.5) ** 2 < 2.0  # P(k) ~ k^-2


def test_two_level_refined_fraction_and_nesting():
    cfg = inputs.two_level_amr(base_level=7, seed=2)
    nf = len(cfg["coords"][1])  # one fine oct per refined base cell
    assert 0.05 <= nf / 128 ** 3 <= 0.10  # refined volume fraction 5-10 %
    # child densities conserve each parent cell's mass
    base = inputs.octs_to_dense(cfg["rho"][0], cfg["coords"][0], 128)
    c = cfg["coords"][1].astype(np.int64)
    assert np.allclose(cfg["rho"][1].mean(axis=1), base[c[:, 0], c[:, 1], c[:, 2]], rtol=1e-12)


def test_batched_patches_structure():
    b = inputs.batched_patches(n_patches=20, n_max=4000, seed=3)
    off, c = b["offsets"], b["coords"].astype(np.int64)
    sizes = np.diff(off)
    assert off[0] == 0 and off[-1] == len(c) and np.all(sizes >= 64) and np.all(sizes <= 4000)
    # each patch inside the central 64^3 of its own 128^3 cube: >= 64 octs apart
    for k in range(20):
        pc = c[off[k]:off[k + 1]]
        cube = np.array([k % 8, (k // 8) % 8, k // 64]) * 128
        assert np.all(pc >= cube + 32) and np.all(pc < cube + 96)
        assert len(np.unique(pc, axis=0)) == len(pc)
    # proper nesting: the 26 neighbours of every patch oct's parent exist
    par = {tuple(x) for x in b["parent_coords"].tolist()}
    for x in c[::17]:
        for d in np.array(np.meshgrid([-1, 0, 1], [-1, 0, 1], [-1, 0, 1])).reshape(3, -1).T:
            assert tuple((x >> 1) + d) in par
    assert b["rho"].shape == (len(c), 8) and np.all(b["rho"] > 0)


def _refine_dense(level, coords, rho_octs, threshold):
    """Brute-force reading of the refinement rule on a dense periodic volume:
    flagged cells, face-dilated among existing cells, kept where all 26
    neighbours exist."""
    off = inputs.child_offsets()
    cells = (2 * coords[:, None, :].astype(np.int64) + off[None, :, :]).reshape(-1, 3)
    size = 1 << level
    exist = np.zeros((size,) * 3, dtype=bool)
    exist[tuple(cells.T)] = True
    flag = np.zeros_like(exist)
    sel = rho_octs.reshape(-1) > threshold
    flag[tuple(cells[sel].T)] = True
    dil = flag.copy()
    for axis in range(3):
        for s in (-1, 1):
            dil |= np.roll(flag, s, axis=axis)
    dil &= exist
    ok = exist.copy()
    for d in np.array(np.meshgrid([-1, 0, 1], [-1, 0, 1], [-1, 0, 1])).reshape(3, -1).T:
        if d.any():
            ok &= np.roll(exist, tuple(-d), axis=(0, 1, 2))
    keep = (dil & ok)[tuple(cells.T)]
    return cells[keep].astype(np.uint32), np.nonzero(keep)[0]


def test_sparse_refinement_matches_dense_rule():
    """The sparse refinement (sorted-key lookups, oct occupancy) selects the
    same cells, in the same order, as the rule applied on dense volumes, down
    a three-level sigma = 2 hierarchy."""
    cfg = inputs.amr_lognormal(5, 3, 2.0, 3)
    assert len(cfg["levels"]) == 4
    for m in range(3):
        lev, c, r = cfg["levels"][m], cfg["coords"][m], cfg["rho"][m]
        got, gi = inputs.refine_cells(lev, c, r, 8.0)
        want, wi = _refine_dense(lev, c, r, 8.0)
        assert np.array_equal(got, want) and np.array_equal(gi, wi)
        assert np.array_equal(got, cfg["coords"][m + 1])
        # children conserve the parent cell's mass
        assert np.allclose(cfg["rho"][m + 1].mean(axis=1), r.reshape(-1)[gi], rtol=1e-12)
