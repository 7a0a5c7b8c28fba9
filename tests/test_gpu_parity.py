"""GPU parity: libcmg.so (through the C ABI) against the CPU oracle on the same
seeded inputs.  Keys, hash lookups, neighbours, father cells and the MG
hierarchy are compared bit-exactly; FP64 fields to 1e-12 relative (the
tolerance fixed for the FP64 path); mixed precision to 1e-10 relative after
refinement against an FP64 oracle converged to 1e-13.

Sizes span several thread blocks with ragged tails; the full-size two-level
workload (128^3 base + refined level) is checked at a fixed cycle count and by
properties that hold at any size."""
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


# ------------------------------------------------------------------ keys

def test_morton_bitexact(cmg, ctx):
    rng = np.random.default_rng(11)
    ijk = rng.integers(0, 1 << 21, size=(100003, 3), dtype=np.uint32)
    k = cmg.cmg_morton_encode(ctx, ijk)
    assert np.array_equal(k, O.morton_encode(ijk))
    assert np.array_equal(cmg.cmg_morton_decode(ctx, k), ijk)
    bad = ijk.copy()
    bad[5, 1] = 1 << 21
    with pytest.raises(cmg.CmgError) as e:
        cmg.cmg_morton_encode(ctx, bad)
    assert e.value.code == cmg.CMG_ERR_KEY_OUT_OF_RANGE


def test_morton_device_memory_path(cmg, ctx):
    import torch
    rng = np.random.default_rng(12)
    ijk = rng.integers(0, 1 << 21, size=(5000, 3), dtype=np.uint32)
    t = torch.from_numpy(ijk).cuda()
    k = cmg.cmg_morton_encode(ctx, t)
    assert k.is_cuda
    assert np.array_equal(k.cpu().numpy(), O.morton_encode(ijk))


@pytest.mark.parametrize("npd,count,level", [(16, 3000, 5), (1 << 20, 70001, 21), (4, 64, 3)])
def test_hash_lookup_bitexact(cmg, ctx, npd, count, level):
    rng = np.random.default_rng(count)
    coords = np.unique(rng.integers(0, npd, size=(count, 3), dtype=np.uint32), axis=0)
    rng.shuffle(coords)
    keys = O.morton_encode(coords)
    G = cmg.cmg_level_build(ctx, level, keys, periodic_mask=7)
    R = O.Level(level, keys, periodic_mask=7)
    assert cmg.cmg_level_hash_capacity(G) == R.hash_capacity
    q = np.concatenate([keys, O.morton_encode(rng.integers(0, npd, size=(count, 3), dtype=np.uint32))])
    assert np.array_equal(cmg.cmg_level_lookup(G, q), R.lookup(q))


def test_build_errors(cmg, ctx):
    k = O.morton_encode(np.array([[0, 0, 0], [1, 0, 0], [0, 0, 0]], dtype=np.uint32))
    with pytest.raises(cmg.CmgError) as e:
        cmg.cmg_level_build(ctx, 3, k)
    assert e.value.code == cmg.CMG_ERR_DUPLICATE_KEY
    with pytest.raises(cmg.CmgError) as e:
        cmg.cmg_level_build(ctx, 2, O.morton_encode(np.array([[2, 0, 0]], dtype=np.uint32)))
    assert e.value.code == cmg.CMG_ERR_KEY_OUT_OF_RANGE
    with pytest.raises(cmg.CmgError) as e:
        cmg.cmg_level_build(ctx, 3, np.array([1 << 63], dtype=np.uint64))
    assert e.value.code == cmg.CMG_ERR_KEY_OUT_OF_RANGE
    with pytest.raises(cmg.CmgError) as e:
        cmg.cmg_level_build(ctx, 0, k[:1])
    assert e.value.code == cmg.CMG_ERR_INVALID_ARG
    # a patch whose coarse-fine stencil leaves its parent patch
    pc = _cube(4, 0.25, 0.75)
    P = cmg.cmg_level_build(ctx, 4, O.morton_encode(pc))
    with pytest.raises(cmg.CmgError) as e:
        cmg.cmg_level_build(ctx, 5, O.morton_encode(_cube(5, 0.25, 0.75)), parent=P)
    assert e.value.code == cmg.CMG_ERR_MISSING_PARENT


def test_empty_level(cmg, ctx):
    G = cmg.cmg_level_build(ctx, 4, np.zeros(0, dtype=np.uint64))
    assert cmg.cmg_level_n_octs(G) == 0
    assert cmg.cmg_level_get_neighbors(G).shape == (0, 7)
    rc, st = cmg.cmg_level_solve(G, tol=1e-10)
    assert rc == cmg.CMG_OK and st["cycles"] == 0


@pytest.mark.parametrize("mode", ["fp64", "mixed", "fft", "pcg"])
def test_uniform_density_gives_zero_phi(cmg, ctx, mode):
    """rho = rho_bar everywhere: the source vanishes and every solve returns
    phi = 0 exactly, with no iteration."""
    coords = inputs.uniform_oct_coords(4)
    G = cmg.cmg_level_build(ctx, 4, O.morton_encode(coords))
    cmg.cmg_level_set_density(G, np.full((len(coords), 8), 2.5), 2.5)
    cmg.cmg_level_set_phi(G, np.random.default_rng(3).standard_normal((len(coords), 8)))
    kw = {"fp64": {}, "mixed": {"precision": cmg.CMG_PREC_MIXED}, "fft": {"precision": cmg.CMG_PREC_FFT},
          "pcg": {"krylov": 1}}[mode]
    rc, st = cmg.cmg_level_solve(G, tol=1e-10, **kw)
    assert rc == cmg.CMG_OK and st["cycles"] == 0
    assert not cmg.cmg_level_get_phi(G).any()


@pytest.mark.parametrize("level", [1, 2])
def test_smallest_periodic_levels(cmg, ctx, level):
    """One oct (the exact 2^3 solve at the top, a one-level hierarchy) and
    eight octs: the discrete solution, as the oracle gives it."""
    coords = inputs.uniform_oct_coords(level)
    rho = 1.0 + np.random.default_rng(level).standard_normal((len(coords), 8))
    G = cmg.cmg_level_build(ctx, level, O.morton_encode(coords))
    R = O.Level(level, O.morton_encode(coords))
    cmg.cmg_level_set_density(G, rho, float(rho.mean()))
    R.set_density(rho, float(rho.mean()))
    rc, st = cmg.cmg_level_solve(G, tol=1e-13)
    R.solve(tol=1e-13)
    assert rc == cmg.CMG_OK
    assert relerr(cmg.cmg_level_get_phi(G), R.get_phi()) <= 1e-12
    if level == 1:
        assert st["cycles"] == 1  # exact in one cycle


def test_single_oct_refined_level(cmg, ctx):
    """A refined level of one oct: all six faces are coarse-fine ghosts."""
    pc = inputs.uniform_oct_coords(4)
    rng = np.random.default_rng(9)
    rho_p = 1.0 + 0.3 * rng.standard_normal((len(pc), 8))
    GP = cmg.cmg_level_build(ctx, 4, O.morton_encode(pc))
    RP = O.Level(4, O.morton_encode(pc))
    for L in (GP, RP):
        (cmg.cmg_level_set_density(L, rho_p, float(rho_p.mean())) if L is GP
         else L.set_density(rho_p, float(rho_p.mean())))
    RP.solve(tol=1e-13)
    cmg.cmg_level_set_phi(GP, RP.get_phi())
    c = np.array([[5, 9, 2]], dtype=np.uint32)
    G = cmg.cmg_level_build(ctx, 5, O.morton_encode(c), parent=GP)
    R = O.Level(5, O.morton_encode(c), parent=RP)
    rho = 1.0 + 0.3 * rng.standard_normal((1, 8))
    cmg.cmg_level_set_density(G, rho, float(rho_p.mean()))
    R.set_density(rho, float(rho_p.mean()))
    assert cmg.cmg_level_get_neighbors(G).tolist() == [[0, -1, -1, -1, -1, -1, -1]]
    rc, st = cmg.cmg_level_solve(G, tol=1e-12)
    R.solve(tol=1e-13)
    assert rc == cmg.CMG_OK
    assert relerr(cmg.cmg_level_get_phi(G), R.get_phi()) <= 1e-11


def test_allocation_failure_injected_on_the_host(cmg, ctx):
    """An allocation that fails (injected on the host, no GPU involved) makes
    the call in progress return CMG_ERR_OOM; the context stays usable and the
    same call afterwards succeeds with correct results -- for a level build
    and for the lazy allocations of FFT, mixed-precision and CG solves."""
    cfg = inputs.two_level_amr(base_level=5, seed=2)
    GB = cmg.cmg_level_build(ctx, 5, O.morton_encode(cfg["coords"][0]))
    cmg.cmg_level_set_density(GB, cfg["rho"][0], 1.0)
    kf = O.morton_encode(cfg["coords"][1])
    try:
        for after in (1, 4, 12):
            cmg.cmg_debug_inject_alloc_failure(after)
            with pytest.raises(cmg.CmgError) as e:
                cmg.cmg_level_build(ctx, 6, kf, parent=GB)
            assert e.value.code == cmg.CMG_ERR_OOM
        cmg.cmg_debug_inject_alloc_failure(0)
        z = np.zeros((cmg.cmg_level_n_octs(GB), 8))
        rc, ref = cmg.cmg_level_solve(GB, tol=1e-12)
        phi_ref = cmg.cmg_level_get_phi(GB)
        for kw in ({"precision": cmg.CMG_PREC_FFT}, {"precision": cmg.CMG_PREC_MIXED}, {"krylov": 1}):
            for after in (1, 2):
                cmg.cmg_level_set_phi(GB, z)
                cmg.cmg_debug_inject_alloc_failure(after)
                rc, st = cmg.cmg_level_solve(GB, tol=1e-12, raise_on_error=False, **kw)
                cmg.cmg_debug_inject_alloc_failure(0)
                assert rc in (cmg.CMG_ERR_OOM, cmg.CMG_OK), (kw, after, rc)
            cmg.cmg_level_set_phi(GB, z)
            rc, st = cmg.cmg_level_solve(GB, tol=1e-12, **kw)
            assert rc == cmg.CMG_OK and relerr(cmg.cmg_level_get_phi(GB), phi_ref) <= 1e-10, kw
        GF = cmg.cmg_level_build(ctx, 6, kf, parent=GB)
        cmg.cmg_level_set_density(GF, cfg["rho"][1], 1.0)
        rc, st = cmg.cmg_level_solve(GF, tol=1e-10)
        assert rc == cmg.CMG_OK
    finally:
        cmg.cmg_debug_inject_alloc_failure(0)
    with pytest.raises(cmg.CmgError) as e:
        cmg.cmg_debug_inject_alloc_failure(-1)
    assert e.value.code == cmg.CMG_ERR_INVALID_ARG


@pytest.mark.parametrize("pmask", [7, 0, 3])
def test_neighbors_bitexact(cmg, ctx, pmask):
    rng = np.random.default_rng(20 + pmask)
    coords = np.unique(rng.integers(0, 32, size=(20000, 3), dtype=np.uint32), axis=0)
    rng.shuffle(coords)
    keys = O.morton_encode(coords)
    G = cmg.cmg_level_build(ctx, 6, keys, periodic_mask=pmask)
    R = O.Level(6, keys, periodic_mask=pmask)
    assert np.array_equal(cmg.cmg_level_get_neighbors(G), R.neighbors())


def _two_level(cmg, ctx, base, seed=2):
    cfg = inputs.two_level_amr(base_level=base, seed=seed)
    kb = cmg.cmg_morton_encode(ctx, cfg["coords"][0])
    kf = cmg.cmg_morton_encode(ctx, cfg["coords"][1])
    GB = cmg.cmg_level_build(ctx, base, kb)
    GF = cmg.cmg_level_build(ctx, base + 1, kf, parent=GB)
    RB = O.Level(base, O.morton_encode(cfg["coords"][0]))
    RF = O.Level(base + 1, O.morton_encode(cfg["coords"][1]), parent=RB)
    return cfg, GB, GF, RB, RF


def test_father_cells_and_hierarchy_bitexact(cmg, ctx):
    cfg, GB, GF, RB, RF = _two_level(cmg, ctx, 5)
    assert np.array_equal(cmg.cmg_level_get_neighbors(GF), RF.neighbors())
    assert np.array_equal(cmg.cmg_level_get_father_cells(GF), RF.father_cells())
    for G, R in ((GB, RB), (GF, RF)):
        assert cmg.cmg_level_mg_depth(G) == R.mg_depth
        for m in range(R.mg_depth):
            n, lev = cmg.cmg_level_mg_info(G, m)
            assert n == R.mg_n_octs(m) and lev == R.mg_lev(m)
            assert np.array_equal(cmg.cmg_level_mg_keys(G, m), R.mg_keys(m))
            assert np.array_equal(cmg.cmg_level_mg_active(G, m), R.mg_active(m))


# ---------------------------------------------------------- single steps

def _random_fields(n, rng):
    return rng.standard_normal((n, 8)), rng.standard_normal((n, 8))


def _set_both(cmg, G, R, m, phi, f):
    cmg.cmg_level_mg_set(G, m, cmg.CMG_FIELD_PHI, phi)
    cmg.cmg_level_mg_set(G, m, cmg.CMG_FIELD_F, f)
    R.mg_set(m, "phi", phi)
    R.mg_set(m, "f", f)
    # the Dirichlet ghosts follow the parent's current phi on both sides
    cmg.cmg_level_mg_step(G, 0, cmg.CMG_OP_GHOSTS)


@pytest.fixture(scope="module")
def two5(cmg, ctx):
    cfg, GB, GF, RB, RF = _two_level(cmg, ctx, 5)
    rng = np.random.default_rng(5)
    phi_b = rng.standard_normal((RB.n, 8))
    cmg.cmg_level_set_phi(GB, phi_b)
    RB.set_phi(phi_b)
    cmg.cmg_level_mg_step(GF, 0, cmg.CMG_OP_GHOSTS)
    return cfg, GB, GF, RB, RF


def test_ghosts_parity(cmg, two5):
    cfg, GB, GF, RB, RF = two5
    g = cmg.cmg_level_get_ghosts(GF)
    r = RF.ghosts()
    assert np.array_equal(np.isnan(g), np.isnan(r))
    ok = ~np.isnan(r)
    assert ok.sum() > 1000
    assert relerr(g[ok], r[ok]) <= 1e-14


@pytest.mark.parametrize("which", ["base", "fine"])
def test_sweep_residual_parity_all_mg_levels(cmg, two5, which):
    cfg, GB, GF, RB, RF = two5
    G, R = (GB, RB) if which == "base" else (GF, RF)
    rng = np.random.default_rng(7)
    for m in range(R.mg_depth):
        n = R.mg_n_octs(m)
        act = R.mg_active(m).astype(bool)
        phi, f = _random_fields(n, rng)
        phi[~act] = 0.0
        _set_both(cmg, G, R, m, phi, f)
        cmg.cmg_level_mg_step(G, m, cmg.CMG_OP_SWEEP, n=2)
        R.rb_sweeps(m, 2, use_ghost=(m == 0))
        got = cmg.cmg_level_mg_get(G, m, cmg.CMG_FIELD_PHI)
        assert relerr(got, R.mg_get(m, "phi")) <= RTOL64, m
        n2 = cmg.cmg_level_mg_step(G, m, cmg.CMG_OP_RESIDUAL)
        r2 = R.residual(m, use_ghost=(m == 0))
        assert abs(n2 - r2) <= 1e-11 * r2, m


def test_residual_field_parity(cmg, two5):
    cfg, GB, GF, RB, RF = two5
    rng = np.random.default_rng(8)
    phi, f = _random_fields(RF.n, rng)
    _set_both(cmg, GF, RF, 0, phi, f)
    r_gpu = cmg.cmg_level_get_residual(GF)
    RF.residual(0, use_ghost=True)
    r_or = RF.mg_get(0, "r")
    assert relerr(r_gpu, r_or) <= RTOL64


@pytest.mark.parametrize("which", ["base", "fine"])
def test_restrict_prolong_coarse_parity(cmg, two5, which):
    cfg, GB, GF, RB, RF = two5
    G, R = (GB, RB) if which == "base" else (GF, RF)
    rng = np.random.default_rng(9)
    for m in range(R.mg_depth - 1):
        n = R.mg_n_octs(m)
        act = R.mg_active(m).astype(bool)
        phi, f = _random_fields(n, rng)
        phi[~act] = 0.0
        _set_both(cmg, G, R, m, phi, f)
        cmg.cmg_level_mg_step(G, m, cmg.CMG_OP_RESTRICT)
        R.residual(m, use_ghost=(m == 0))
        R.restrict(m)
        # only active coarse cells carry a restricted residual (inactive ones
        # are never read)
        cact = R.mg_active(m + 1).astype(bool)
        cf = cmg.cmg_level_mg_get(G, m + 1, cmg.CMG_FIELD_F)
        assert relerr(cf[cact], R.mg_get(m + 1, "f")[cact]) <= 1e-11, m
        assert np.all(cmg.cmg_level_mg_get(G, m + 1, cmg.CMG_FIELD_PHI) == 0.0)
        cact = R.mg_active(m + 1).astype(bool)
        e = rng.standard_normal((R.mg_n_octs(m + 1), 8))
        e[~cact] = 0.0
        cmg.cmg_level_mg_set(G, m + 1, cmg.CMG_FIELD_PHI, e)
        R.mg_set(m + 1, "phi", e)
        cmg.cmg_level_mg_step(G, m, cmg.CMG_OP_PROLONG)
        R.prolong(m)
        assert relerr(cmg.cmg_level_mg_get(G, m, cmg.CMG_FIELD_PHI), R.mg_get(m, "phi")) <= RTOL64, m
    last = R.mg_depth - 1
    f = rng.standard_normal((R.mg_n_octs(last), 8))
    f[~R.mg_active(last).astype(bool)] = 0.0
    if which == "base":
        f -= f.mean()
    _set_both(cmg, G, R, last, np.zeros_like(f), f)
    cmg.cmg_level_mg_step(G, last, cmg.CMG_OP_COARSE, n=32)
    R.coarse_solve(32)
    assert relerr(cmg.cmg_level_mg_get(G, last, cmg.CMG_FIELD_PHI), R.mg_get(last, "phi")) <= RTOL64


# ------------------------------------------------------------ V-cycles

def _solve_pair(cmg, G, R, fixed=0, tol=1e-10, **kw):
    rc, st = cmg.cmg_level_solve(G, tol=tol, fixed_cycles=fixed, **kw)
    R.solve(tol=tol, fixed_cycles=fixed)
    return st


def test_config1_periodic_32cube_solve(cmg, ctx):
    cfg = inputs.periodic_grf_level(5, seed=1)
    keys = cmg.cmg_morton_encode(ctx, cfg["coords"][0])
    G = cmg.cmg_level_build(ctx, 5, keys)
    R = O.Level(5, O.morton_encode(cfg["coords"][0]))
    cmg.cmg_level_set_density(G, cfg["rho"][0], 1.0)
    R.set_density(cfg["rho"][0], 1.0)
    rc, st = cmg.cmg_level_solve(G, tol=1e-10)
    ro, so = R.solve(tol=1e-10)
    assert st["cycles"] == so["cycles"]
    np.testing.assert_allclose(st["rel_history"], so["rel_history"], rtol=1e-4)
    phi = cmg.cmg_level_get_phi(G)
    assert relerr(phi, R.get_phi()) <= RTOL64
    assert st["rel_final"] <= 1e-10
    assert abs(phi.mean()) <= 1e-14 * np.abs(phi).max()


@pytest.mark.parametrize("base", [5, 6])
def test_two_level_fixed_cycles_and_converged(cmg, ctx, base):
    cfg, GB, GF, RB, RF = _two_level(cmg, ctx, base)
    for G, R, rho in ((GB, RB, cfg["rho"][0]), (GF, RF, cfg["rho"][1])):
        cmg.cmg_level_set_density(G, rho, 1.0)
        R.set_density(rho, 1.0)
    _solve_pair(cmg, GB, RB, fixed=3)
    assert relerr(cmg.cmg_level_get_phi(GB), RB.get_phi()) <= RTOL64
    _solve_pair(cmg, GF, RF, fixed=3)
    assert relerr(cmg.cmg_level_get_phi(GF), RF.get_phi()) <= RTOL64
    # converged to 1e-10 from zero on both sides
    for G, R in ((GB, RB), (GF, RF)):
        z = np.zeros((R.n, 8))
        cmg.cmg_level_set_phi(G, z)
        R.set_phi(z)
        st = _solve_pair(cmg, G, R, tol=1e-10)
        assert relerr(cmg.cmg_level_get_phi(G), R.get_phi()) <= RTOL64
        assert st["rel_final"] <= 1e-10


def test_two_level_full_size_128(cmg, ctx):
    """The 128^3 two-level workload: two cycles against the oracle, then the
    converged GPU solution checked by an independent residual evaluation."""
    cfg, GB, GF, RB, RF = _two_level(cmg, ctx, 7)
    for G, R, rho in ((GB, RB, cfg["rho"][0]), (GF, RF, cfg["rho"][1])):
        cmg.cmg_level_set_density(G, rho, 1.0)
        R.set_density(rho, 1.0)
    _solve_pair(cmg, GB, RB, fixed=2)
    assert relerr(cmg.cmg_level_get_phi(GB), RB.get_phi()) <= RTOL64
    _solve_pair(cmg, GF, RF, fixed=2)
    assert relerr(cmg.cmg_level_get_phi(GF), RF.get_phi()) <= RTOL64
    # converged GPU solve; residual recomputed by the oracle
    for G, R in ((GB, RB), (GF, RF)):
        rc, st = cmg.cmg_level_solve(G, tol=1e-10)
        assert st["rel_final"] <= 1e-10
        R.set_phi(cmg.cmg_level_get_phi(G))
        n2 = R.residual(0, use_ghost=True)
        assert np.sqrt(n2) <= 1.0001e-10 * st["norm0"]


@pytest.mark.parametrize("inner", [1, 2, 3])
def test_mixed_precision_matches_fp64(cmg, ctx, inner):
    """FP32 V-cycles (1 to 3 per refinement step) inside FP64 refinement reach
    the FP64 solution: at the stopping residual 1e-11 phi agrees with the
    oracle converged to 1e-13 to 1e-10 relative, and refinement keeps going
    below FP32 round-off."""
    cfg, GB, GF, RB, RF = _two_level(cmg, ctx, 6)
    for G, R, rho in ((GB, RB, cfg["rho"][0]), (GF, RF, cfg["rho"][1])):
        cmg.cmg_level_set_density(G, rho, 1.0)
        R.set_density(rho, 1.0)
        R.solve(tol=1e-13)
        rc, st = cmg.cmg_level_solve(G, tol=1e-11, precision=cmg.CMG_PREC_MIXED, inner_cycles=inner)
        assert st["rel_final"] <= 1e-11
        assert relerr(cmg.cmg_level_get_phi(G), R.get_phi()) <= RTOL_MIXED
        rc, st = cmg.cmg_level_solve(G, tol=1e-13, precision=cmg.CMG_PREC_MIXED, inner_cycles=inner)
        assert st["rel_final"] <= 1e-13
        # the parent phi the fine level sees is the GPU's own mixed solution
        if G is GB:
            RB.set_phi(cmg.cmg_level_get_phi(GB))


def test_status_codes(cmg, ctx):
    cfg = inputs.periodic_grf_level(4, seed=1)
    G = cmg.cmg_level_build(ctx, 4, cmg.cmg_morton_encode(ctx, cfg["coords"][0]))
    cmg.cmg_level_set_density(G, cfg["rho"][0], 1.0)
    rc, st = cmg.cmg_level_solve(G, tol=1e-10, max_cycles=2, raise_on_error=False)
    assert rc == cmg.CMG_ERR_NOT_CONVERGED and st["cycles"] == 2
    rho = cfg["rho"][0].copy()
    rho[3, 2] = np.nan
    cmg.cmg_level_set_density(G, rho, 1.0)
    rc, st = cmg.cmg_level_solve(G, tol=1e-10, raise_on_error=False)
    assert rc == cmg.CMG_ERR_DIVERGED
    with pytest.raises(cmg.CmgError) as e:
        cmg.cmg_level_solve(G, tol=1e-10, n_pre=-1)
    assert e.value.code == cmg.CMG_ERR_INVALID_ARG


def test_device_arrays_match_host_arrays(cmg, ctx):
    import torch
    cfg = inputs.periodic_grf_level(5, seed=1)
    keys = torch.from_numpy(O.morton_encode(cfg["coords"][0])).cuda()
    G = cmg.cmg_level_build(ctx, 5, keys)
    cmg.cmg_level_set_density(G, torch.from_numpy(cfg["rho"][0]).cuda(), 1.0)
    cmg.cmg_level_solve(G, tol=1e-10)
    phi_d = cmg.cmg_level_get_phi(G, device=True)
    H = cmg.cmg_level_build(ctx, 5, O.morton_encode(cfg["coords"][0]))
    cmg.cmg_level_set_density(H, cfg["rho"][0], 1.0)
    cmg.cmg_level_solve(H, tol=1e-10)
    assert np.array_equal(phi_d.cpu().numpy(), cmg.cmg_level_get_phi(H))


@pytest.mark.parametrize("precision", [0, 1])
def test_tail_schedule_matches_per_operation_launches(cmg, ctx, precision):
    """The tail kernels (one CTA for the smallest levels, a cooperative grid
    launch above; one thread per oct, or per cell on small FP64 levels) run
    the same arithmetic, in the same order, as the one-launch-per-operation
    path: the schedule must not change a bit of phi.  Tails from 64 octs (one
    CTA in FP64 and FP32), 512 (grid in FP64 with the levels of at most 64
    octs on CTA 0; one CTA in FP32), 4096 (grid in FP64, one CTA in FP32) and
    the whole hierarchy below the level itself (grid)."""
    cfg, GB, GF, RB, RF = _two_level(cmg, ctx, 6)
    out = {}
    tails = (0, 64, 512, 4096, 1 << 20)
    for tail in tails:
        for G, rho in ((GB, cfg["rho"][0]), (GF, cfg["rho"][1])):
            cmg.cmg_level_set_schedule(G, tail, tail)
            cmg.cmg_level_set_density(G, rho, 1.0)
            cmg.cmg_level_set_phi(G, np.zeros((cmg.cmg_level_n_octs(G), 8)))
            rc, st = cmg.cmg_level_solve(G, tol=1e-10, fixed_cycles=4, precision=precision)
            out[(tail, G is GB)] = cmg.cmg_level_get_phi(G)
    for tail in tails[1:]:
        for base in (True, False):
            assert np.array_equal(out[(tail, base)], out[(0, base)]), (tail, base)


@pytest.mark.parametrize("n_post", [1, 2])
def test_colour1_residual_is_exactly_zero_after_a_cycle(cmg, ctx, n_post):
    """An FP64 cycle ends with a colour-1 pass on the top level, which wrote
    fma(s, 1/6, g) at every colour-1 cell from the colour-0 values that the
    residual reads, summed in the same order: each colour-1 residual is
    exactly 0.0 while the colour-0 ones are not.  The stopping residual and
    the V-cycle's restrictions skip those stencils on this ground (bit-
    identical results); a change to either kernel's summation order breaks
    this test first.  Refined level (no mean subtraction after the solve)."""
    cfg, GB, GF, RB, RF = _two_level(cmg, ctx, 6)
    for G, rho in ((GB, cfg["rho"][0]), (GF, cfg["rho"][1])):
        cmg.cmg_level_set_density(G, rho, 1.0)
        cmg.cmg_level_set_phi(G, np.zeros((cmg.cmg_level_n_octs(G), 8)))
    cmg.cmg_level_solve(GB, tol=1e-10)
    cmg.cmg_level_solve(GF, fixed_cycles=2, n_post=n_post)
    r = cmg.cmg_level_get_residual(GF)
    odd, even = [1, 2, 4, 7], [0, 3, 5, 6]
    assert np.all(r[:, odd] == 0.0)
    assert np.count_nonzero(r[:, even]) > 0.9 * r[:, even].size


@pytest.mark.parametrize("n_pre,n_post", [(0, 2), (2, 0), (1, 1), (1, 3)])
def test_smoothing_counts_match_oracle(cmg, ctx, n_pre, n_post):
    """V(n_pre, n_post) cycles other than V(2,2).  With n_pre = 0 no colour-1
    pass precedes the restriction, which then evaluates every residual (and
    the coarse phi is zeroed); with n_post = 0 the prolongation corrects every
    cell and the stopping residual is evaluated in full.  Fixed FP64 cycles
    against the oracle (1e-12), both levels with the same parent phi; mixed
    precision refined to 1e-12 against the oracle converged to 1e-13."""
    cfg, GB, GF, RB, RF = _two_level(cmg, ctx, 6)
    for k, (G, R, rho) in enumerate(((GB, RB, cfg["rho"][0]), (GF, RF, cfg["rho"][1]))):
        if k == 1:
            cmg.cmg_level_set_phi(GB, RB.get_phi())
        cmg.cmg_level_set_density(G, rho, 1.0)
        R.set_density(rho, 1.0)
        z = np.zeros((R.n, 8))
        cmg.cmg_level_set_phi(G, z)
        R.set_phi(z)
        rc, st = cmg.cmg_level_solve(G, fixed_cycles=3, n_pre=n_pre, n_post=n_post)
        ro, so = R.solve(fixed_cycles=3, n_pre=n_pre, n_post=n_post)
        assert relerr(cmg.cmg_level_get_phi(G), R.get_phi()) <= RTOL64, k
        np.testing.assert_allclose(st["rel_history"], so["rel_history"], rtol=1e-9)
        R.solve(tol=1e-13, n_pre=n_pre, n_post=n_post)
        cmg.cmg_level_set_phi(G, z)
        rc, st = cmg.cmg_level_solve(G, tol=1e-12, n_pre=n_pre, n_post=n_post, precision=cmg.CMG_PREC_MIXED)
        assert rc == cmg.CMG_OK and st["rel_final"] <= 1e-12, k
        assert relerr(cmg.cmg_level_get_phi(G), R.get_phi()) <= 1e-10, k


def test_queued_solves_match_blocking_solves(cmg, ctx):
    """cmg_level_solve_async + cmg_level_solve_wait on both levels of the
    two-level workload (the fine level queued behind its parent, whose phi it
    reads in stream order) give the blocking solves' phi and statistics
    bit-for-bit; waiting with nothing queued and queueing twice are errors."""
    cfg, GB, GF, RB, RF = _two_level(cmg, ctx, 6)
    out = {}
    for mode in ("blocking", "queued"):
        for G, rho in ((GB, cfg["rho"][0]), (GF, cfg["rho"][1])):
            cmg.cmg_level_set_density(G, rho, 1.0)
            cmg.cmg_level_set_phi(G, np.zeros((cmg.cmg_level_n_octs(G), 8)))
        if mode == "blocking":
            sts = [cmg.cmg_level_solve(G, tol=1e-10)[1] for G in (GB, GF)]
        else:
            for G in (GB, GF):
                cmg.cmg_level_solve_async(G, tol=1e-10)
            sts = [cmg.cmg_level_solve_wait(G)[1] for G in (GB, GF)]
        out[mode] = ([cmg.cmg_level_get_phi(G) for G in (GB, GF)], sts)
    for a, b in zip(out["blocking"][0], out["queued"][0]):
        assert np.array_equal(a, b)
    for a, b in zip(out["blocking"][1], out["queued"][1]):
        assert a["cycles"] == b["cycles"] and a["rel_history"] == b["rel_history"]
    with pytest.raises(cmg.CmgError) as e:
        cmg.cmg_level_solve_wait(GB)
    assert e.value.code == cmg.CMG_ERR_INVALID_ARG
    cmg.cmg_level_solve_async(GB, tol=1e-10)
    with pytest.raises(cmg.CmgError) as e:
        cmg.cmg_level_solve_async(GB, tol=1e-10)
    assert e.value.code == cmg.CMG_ERR_INVALID_ARG
    rc, st = cmg.cmg_level_solve_wait(GB)
    assert rc == cmg.CMG_OK


def test_async_read_back_overlapping_the_next_solve(cmg, ctx):
    """Host-memory upload and read-back on the copy streams: the base level's
    density upload, solve and queued phi read-back, then the fine level's
    (its upload overlapping the base solve, the base read-back overlapping
    the fine solve) give, after cmg_ctx_synchronize, the phi of blocking
    calls bit-for-bit, in pinned and in pageable host buffers; a second
    queued read-back of the same staging buffer waits for the first."""
    import torch
    cfg, GB, GF, RB, RF = _two_level(cmg, ctx, 6)
    z = [np.zeros((cmg.cmg_level_n_octs(G), 8)) for G in (GB, GF)]
    for G, rho, zz in zip((GB, GF), cfg["rho"], z):
        cmg.cmg_level_set_phi(G, zz)
        cmg.cmg_level_set_density(G, rho, 1.0)
        cmg.cmg_level_solve(G, tol=1e-10)
    ref = [cmg.cmg_level_get_phi(G) for G in (GB, GF)]
    for pinned in (True, False):
        rho = [torch.from_numpy(r).pin_memory().numpy() if pinned else r.copy() for r in cfg["rho"]]
        out = [torch.empty(r.shape, dtype=torch.float64).pin_memory().numpy() if pinned else np.empty(r.shape)
               for r in ref]
        for G, r, zz, o in zip((GB, GF), rho, z, out):
            cmg.cmg_level_set_phi(G, zz)
            cmg.cmg_level_set_density(G, r, 1.0)
            cmg.cmg_level_solve_async(G, tol=1e-10)
            cmg.cmg_level_get_phi_async(G, out=o)
        for G in (GB, GF):
            rc, st = cmg.cmg_level_solve_wait(G)
            assert rc == cmg.CMG_OK
        cmg.cmg_ctx_synchronize(ctx)
        for o, r in zip(out, ref):
            assert np.array_equal(o, r), pinned


def test_grid_tail_barrier_timeout_returns_status(cmg, ctx):
    """A grid-tail barrier wait that runs out of spin budget ends the launch
    and the solve with CMG_ERR_TIMEOUT; the context stays usable and the next
    solve with the default budget converges."""
    cfg, GB, GF, RB, RF = _two_level(cmg, ctx, 6)
    cmg.cmg_level_set_schedule(GB, 1 << 20, 1 << 20)
    cmg.cmg_level_set_density(GB, cfg["rho"][0], 1.0)
    z = np.zeros((cmg.cmg_level_n_octs(GB), 8))
    cmg.cmg_level_set_spin_budget(GB, 0)
    cmg.cmg_level_set_phi(GB, z)
    rc, st = cmg.cmg_level_solve(GB, tol=1e-10, raise_on_error=False)
    assert rc == cmg.CMG_ERR_TIMEOUT
    cmg.cmg_level_set_spin_budget(GB, 1 << 30)
    cmg.cmg_level_set_phi(GB, z)
    rc, st = cmg.cmg_level_solve(GB, tol=1e-10)
    assert rc == cmg.CMG_OK and st["rel_final"] <= 1e-10
    with pytest.raises(cmg.CmgError) as e:
        cmg.cmg_level_set_spin_budget(GB, -1)
    assert e.value.code == cmg.CMG_ERR_INVALID_ARG


def _cube(level, lo, hi):
    npd = 1 << (level - 1)
    r = np.arange(int(round(lo * npd)), int(round(hi * npd)))
    z, y, x = np.meshgrid(r, r, r, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], 1).astype(np.uint32)
