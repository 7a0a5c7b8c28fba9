"""128-bit Morton keys on the GPU (Sec. 4.2: B = 42, levels up to 43) against
the oracle: keys, hash lookups, neighbours, father cells and the multigrid
hierarchy bit-exactly, and the level solve to the FP64 / mixed-precision bars,
on a zoom chain from a periodic 16^3 base to level 30 (levels 23..30 are out
of reach of 64-bit keys).  Where coordinates fit 21 bits the 128-bit build
must reproduce the 64-bit one exactly."""
import numpy as np
import pytest

import oracle as O
from paper_2604_06035_gb300 import inputs

pytestmark = pytest.mark.gpu

RTOL64 = 1e-12
RTOL_MIXED = 1e-10


@pytest.fixture(scope="module")
def cmg():
    import __graft_entry__ as ge
    ge.build()
    from paper_2604_06035_gb300 import cmg as _c
    return _c


@pytest.fixture(scope="module")
def ctx(cmg):
    c = cmg.cmg_ctx_create(0)
    yield c
    import gc
    gc.collect()
    cmg.cmg_ctx_destroy(c)


def relerr(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def test_morton128_bitexact(cmg, ctx):
    rng = np.random.default_rng(21)
    ijk = rng.integers(0, 1 << 42, size=(100003, 3), dtype=np.uint64)
    ijk[:3] = [[(1 << 21) - 1, 1 << 21, 0], [(1 << 42) - 1] * 3, [0, 0, 0]]
    k = cmg.cmg_morton_encode128(ctx, ijk)
    assert np.array_equal(k, O.morton_encode128(ijk))
    assert np.array_equal(cmg.cmg_morton_decode128(ctx, k), ijk)
    bad = ijk[:10].copy()
    bad[4, 2] = 1 << 42
    with pytest.raises(cmg.CmgError) as e:
        cmg.cmg_morton_encode128(ctx, bad)
    assert e.value.code == cmg.CMG_ERR_KEY_OUT_OF_RANGE


@pytest.fixture(scope="module")
def zoom(cmg, ctx):
    cfg = inputs.deep_zoom(top_level=30)
    G, R = [], []
    for lev, c, rho in zip(cfg["levels"], cfg["coords"], cfg["rho"]):
        keys = O.morton_encode128(c)
        G.append(cmg.cmg_level_build128(ctx, lev, keys, parent=G[-1] if G else None))
        R.append(O.Level(lev, keys, parent=R[-1] if R else None))
        cmg.cmg_level_set_density(G[-1], rho, cfg["rho_bar"])
        R[-1].set_density(rho, cfg["rho_bar"])
    return cfg, G, R


def test_zoom_structure_bitexact(cmg, zoom):
    cfg, G, R = zoom
    for lev, c, g, r in zip(cfg["levels"], cfg["coords"], G, R):
        assert cmg.cmg_level_key_bits(g) == 128
        keys = O.morton_encode128(c)
        assert np.array_equal(cmg.cmg_level_lookup128(g, keys), np.arange(len(c)))
        q = O.morton_encode128(c + np.uint64(3))
        assert np.array_equal(cmg.cmg_level_lookup128(g, q), r.lookup(q))
        assert np.array_equal(cmg.cmg_level_get_neighbors(g), r.neighbors()), lev
        assert np.array_equal(cmg.cmg_level_get_father_cells(g), r.father_cells()), lev
        assert cmg.cmg_level_mg_depth(g) == r.mg_depth, lev
        for m in range(r.mg_depth):
            assert np.array_equal(cmg.cmg_level_mg_keys128(g, m), r.mg_keys(m)), (lev, m)
            assert np.array_equal(cmg.cmg_level_mg_active(g, m), r.mg_active(m)), (lev, m)


def test_zoom_solves_match_oracle(cmg, zoom):
    cfg, G, R = zoom
    for k, (g, r) in enumerate(zip(G, R)):
        # the same parent phi on both sides: the oracle's converged one
        if k > 0:
            cmg.cmg_level_set_phi(G[k - 1], R[k - 1].get_phi())
        z = np.zeros((r.n, 8))
        cmg.cmg_level_set_phi(g, z)
        r.set_phi(z)
        rc, st = cmg.cmg_level_solve(g, fixed_cycles=3)
        ro, so = r.solve(fixed_cycles=3)
        assert relerr(cmg.cmg_level_get_phi(g), r.get_phi()) <= RTOL64, cfg["levels"][k]
        r.solve(tol=1e-13)
        cmg.cmg_level_set_phi(g, z)
        rc, st = cmg.cmg_level_solve(g, tol=1e-12, precision=cmg.CMG_PREC_MIXED)
        assert rc == cmg.CMG_OK and st["rel_final"] <= 1e-12
        assert relerr(cmg.cmg_level_get_phi(g), r.get_phi()) <= RTOL_MIXED, cfg["levels"][k]


def test_128bit_levels_reproduce_64bit_levels(cmg, ctx):
    cfg = inputs.two_level_amr(base_level=6, seed=2)
    A, W = [], []
    for lev, c, rho in zip(cfg["levels"], cfg["coords"], cfg["rho"]):
        A.append(cmg.cmg_level_build(ctx, lev, O.morton_encode(c), parent=A[-1] if A else None))
        W.append(cmg.cmg_level_build128(ctx, lev, O.morton_encode128(c.astype(np.uint64)),
                                        parent=W[-1] if W else None))
        for L in (A[-1], W[-1]):
            cmg.cmg_level_set_density(L, rho, 1.0)
            cmg.cmg_level_solve(L, tol=1e-10)
        assert np.array_equal(cmg.cmg_level_get_neighbors(A[-1]), cmg.cmg_level_get_neighbors(W[-1]))
        assert np.array_equal(cmg.cmg_level_get_phi(A[-1]), cmg.cmg_level_get_phi(W[-1])), lev
    # the FFT solve reads a 128-bit base level's low key words
    rc, st = cmg.cmg_level_solve(W[0], tol=1e-11, precision=cmg.CMG_PREC_FFT)
    assert rc == cmg.CMG_OK and st["rel_final"] <= 1e-11


def test_key_width_errors(cmg, ctx, zoom):
    cfg, G, R = zoom
    c = cfg["coords"][1]
    with pytest.raises(cmg.CmgError) as e:  # 64-bit child of a 128-bit parent
        cmg.cmg_level_build(ctx, 5, O.morton_encode(c.astype(np.uint32)), parent=G[0])
    assert e.value.code == cmg.CMG_ERR_INVALID_ARG
    with pytest.raises(cmg.CmgError) as e:
        cmg.cmg_level_lookup(G[-1], np.zeros(1, dtype=np.uint64))
    assert e.value.code == cmg.CMG_ERR_INVALID_ARG
    one = O.morton_encode128(np.zeros((1, 3), dtype=np.uint64))
    with pytest.raises(cmg.CmgError) as e:
        cmg.cmg_level_build128(ctx, 44, one, periodic_mask=0)
    assert e.value.code == cmg.CMG_ERR_INVALID_ARG
    with pytest.raises(cmg.CmgError) as e:
        cmg.cmg_level_build(ctx, 23, np.zeros(1, dtype=np.uint64), periodic_mask=0)
    assert e.value.code == cmg.CMG_ERR_INVALID_ARG
    far = O.morton_encode128(np.array([[1 << 29, 0, 0]], dtype=np.uint64))
    with pytest.raises(cmg.CmgError) as e:
        cmg.cmg_level_build128(ctx, 30, far, periodic_mask=0)
    assert e.value.code == cmg.CMG_ERR_KEY_OUT_OF_RANGE
