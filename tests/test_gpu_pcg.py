"""Multigrid-preconditioned conjugate gradients (krylov = 1) against the
oracle's PCG on the same inputs.

Both run the same flexible CG with one V-cycle per iteration as the
preconditioner; only the order of the floating-point reductions differs,
which perturbs alpha and beta at the 1e-16 level.  So iteration histories
agree to 1e-9 relative above an absolute floor of 1e-15 (a relative residual
near 1e-13 carries the reductions' rounding, ~1e-16 of the initial norm),
phi after a fixed number of iterations to 1e-11 and converged phi to the
FP64 bar (1e-12 relative, plus the stopping residual's own spread)."""
import numpy as np
import pytest

import oracle as O
from paper_2604_06035_gb300 import inputs
from tests import dense_ref as DR

pytestmark = pytest.mark.gpu


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


def test_pcg_periodic_matches_oracle_and_exact(cmg, ctx):
    cfg = inputs.periodic_grf_level(5, rms=0.5, seed=1)
    coords = cfg["coords"][0]
    G = cmg.cmg_level_build(ctx, 5, cmg.cmg_morton_encode(ctx, coords))
    R = O.Level(5, O.morton_encode(coords))
    cmg.cmg_level_set_density(G, cfg["rho"][0], 1.0)
    R.set_density(cfg["rho"][0], 1.0)
    rc, st = cmg.cmg_level_solve(G, tol=1e-12, krylov=1)
    ro, so = R.solve_pcg(tol=1e-12)
    assert st["cycles"] == so["cycles"]
    np.testing.assert_allclose(st["rel_history"], so["rel_history"], rtol=1e-9, atol=1e-15)
    phi = cmg.cmg_level_get_phi(G)
    assert relerr(phi, R.get_phi()) <= 1e-12
    f = inputs.octs_to_dense(cfg["rho"][0] - 1.0, coords, 32)
    exact = inputs.dense_to_octs(DR.fft_solve(f, 1.0 / 32), coords)
    assert relerr(phi, exact) <= 1e-10
    assert abs(phi.mean()) <= 1e-14 * np.abs(phi).max()


@pytest.mark.parametrize("base", [5, 6])
def test_pcg_refined_level_matches_oracle(cmg, ctx, base):
    cfg = inputs.two_level_amr(base_level=base, seed=2)
    GB = cmg.cmg_level_build(ctx, base, cmg.cmg_morton_encode(ctx, cfg["coords"][0]))
    GF = cmg.cmg_level_build(ctx, base + 1, cmg.cmg_morton_encode(ctx, cfg["coords"][1]), parent=GB)
    RB = O.Level(base, O.morton_encode(cfg["coords"][0]))
    RF = O.Level(base + 1, O.morton_encode(cfg["coords"][1]), parent=RB)
    for G, R, rho in ((GB, RB, cfg["rho"][0]), (GF, RF, cfg["rho"][1])):
        cmg.cmg_level_set_density(G, rho, 1.0)
        R.set_density(rho, 1.0)
    RB.solve(tol=1e-13)
    cmg.cmg_level_set_phi(GB, RB.get_phi())  # the same parent values on both sides
    # a fixed number of iterations
    rc, st = cmg.cmg_level_solve(GF, fixed_cycles=3, krylov=1)
    ro, so = RF.solve_pcg(fixed_cycles=3)
    np.testing.assert_allclose(st["rel_history"], so["rel_history"], rtol=1e-9, atol=1e-15)
    assert relerr(cmg.cmg_level_get_phi(GF), RF.get_phi()) <= 1e-11
    # converged, from zero on both sides
    z = np.zeros((RF.n, 8))
    cmg.cmg_level_set_phi(GF, z)
    RF.set_phi(z)
    rc, st = cmg.cmg_level_solve(GF, tol=1e-12, krylov=1)
    ro, so = RF.solve_pcg(tol=1e-12)
    assert abs(st["cycles"] - so["cycles"]) <= 1
    assert relerr(cmg.cmg_level_get_phi(GF), RF.get_phi()) <= 1e-11
    # fewer iterations than the stationary V-cycle iteration
    cmg.cmg_level_set_phi(GF, z)
    rc, st_mg = cmg.cmg_level_solve(GF, tol=1e-12)
    assert st["cycles"] < st_mg["cycles"]
    # the level is left as a solve leaves it: the source restored, the ghosts
    # refilled, phi converged (a stationary solve from it has nothing to do)
    cmg.cmg_level_set_phi(GF, RF.get_phi())
    rc, st2 = cmg.cmg_level_solve(GF, tol=1e-11)
    assert st2["cycles"] == 0 and st2["rel_initial"] <= 1e-11


@pytest.mark.parametrize("base", [5, 6])
def test_pcg_mixed_precision_preconditioner(cmg, ctx, base):
    """krylov = 1 with MIXED precision: FP32 V-cycles on r / ||r|| as the
    (inexact) preconditioner of the FP64 flexible CG.  Refined to rel.
    residual 1e-12 it agrees with the oracle converged to 1e-13 to 1e-10 (the
    mixed-precision bar), in fewer iterations than the stationary mixed
    iteration, and leaves the level as a solve leaves it."""
    cfg = inputs.two_level_amr(base_level=base, seed=2)
    GB = cmg.cmg_level_build(ctx, base, cmg.cmg_morton_encode(ctx, cfg["coords"][0]))
    GF = cmg.cmg_level_build(ctx, base + 1, cmg.cmg_morton_encode(ctx, cfg["coords"][1]), parent=GB)
    RB = O.Level(base, O.morton_encode(cfg["coords"][0]))
    RF = O.Level(base + 1, O.morton_encode(cfg["coords"][1]), parent=RB)
    for G, R, rho in ((GB, RB, cfg["rho"][0]), (GF, RF, cfg["rho"][1])):
        cmg.cmg_level_set_density(G, rho, 1.0)
        R.set_density(rho, 1.0)
    RB.solve(tol=1e-13)
    cmg.cmg_level_set_phi(GB, RB.get_phi())
    RF.solve(tol=1e-13)
    for G, R in ((GB, RB), (GF, RF)):
        z = np.zeros((R.n, 8))
        cmg.cmg_level_set_phi(G, z)
        rc, st_mg = cmg.cmg_level_solve(G, tol=1e-12, precision=cmg.CMG_PREC_MIXED)
        cmg.cmg_level_set_phi(G, z)
        rc, st = cmg.cmg_level_solve(G, tol=1e-12, precision=cmg.CMG_PREC_MIXED, krylov=1)
        assert rc == cmg.CMG_OK and st["rel_final"] <= 1e-12
        assert st["cycles"] <= st_mg["cycles"]
        assert relerr(cmg.cmg_level_get_phi(G), R.get_phi()) <= 1e-10
        rc, st2 = cmg.cmg_level_solve(G, tol=1e-11)
        assert st2["cycles"] == 0
        if G is GB:
            cmg.cmg_level_set_phi(GB, RB.get_phi())


def test_pcg_rejects_fft_and_bad_values(cmg, ctx):
    cfg = inputs.periodic_grf_level(4, seed=1)
    G = cmg.cmg_level_build(ctx, 4, cmg.cmg_morton_encode(ctx, cfg["coords"][0]))
    cmg.cmg_level_set_density(G, cfg["rho"][0], 1.0)
    with pytest.raises(cmg.CmgError) as e:
        cmg.cmg_level_solve(G, tol=1e-10, krylov=1, precision=cmg.CMG_PREC_FFT)
    assert e.value.code == cmg.CMG_ERR_INVALID_ARG
    with pytest.raises(cmg.CmgError):
        cmg.cmg_level_solve(G, tol=1e-10, krylov=2)
