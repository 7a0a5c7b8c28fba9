"""FFT solve of full periodic levels (FP32 FFT direct solve of the correction
equation inside the FP64 iterative refinement) against the oracle.

The transform error is FP32 (a few 1e-7 relative per step), so each
refinement step gains ~6 digits: the solve must reach the requested FP64
tolerance in a handful of steps and agree with the oracle converged to 1e-13
to 1e-10 relative, the mixed-precision bar.  The oracle here is the FP64
multigrid solve and, independently, the exact solution of the discrete
operator by numpy's FP64 FFT."""
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


@pytest.mark.parametrize("level", [2, 4, 5, 6])
def test_fft_solve_matches_oracle(cmg, ctx, level):
    cfg = inputs.periodic_grf_level(level, rms=0.5, seed=3)
    coords = cfg["coords"][0]
    G = cmg.cmg_level_build(ctx, level, cmg.cmg_morton_encode(ctx, coords))
    R = O.Level(level, O.morton_encode(coords))
    rho = cfg["rho"][0]
    cmg.cmg_level_set_density(G, rho, 1.0)
    R.set_density(rho, 1.0)
    R.solve(tol=1e-13)
    rc, st = cmg.cmg_level_solve(G, tol=1e-11, precision=cmg.CMG_PREC_FFT)
    assert rc == cmg.CMG_OK and st["rel_final"] <= 1e-11
    assert st["cycles"] <= 4
    phi = cmg.cmg_level_get_phi(G)
    assert relerr(phi, R.get_phi()) <= 1e-10
    # the exact discrete solution (numpy FP64 FFT of the dense source)
    n = 1 << level
    f = inputs.octs_to_dense(rho - 1.0, coords, n)
    exact = inputs.dense_to_octs(DR.fft_solve(f, 1.0 / n), coords)
    assert relerr(phi, exact) <= 1e-10
    # refinement keeps going below FP32 round-off
    rc, st = cmg.cmg_level_solve(G, tol=1e-13, precision=cmg.CMG_PREC_FFT)
    assert st["rel_final"] <= 1e-13
    assert relerr(cmg.cmg_level_get_phi(G), exact) <= 1e-12


def test_fft_solve_lognormal_base_128(cmg, ctx):
    """The two-level workload's 128^3 lognormal base (sigma 1.5): FFT solve
    against the GPU FP64 multigrid solution, residual re-evaluated by the
    oracle."""
    cfg = inputs.two_level_amr(base_level=7, seed=2)
    coords = cfg["coords"][0]
    G = cmg.cmg_level_build(ctx, 7, cmg.cmg_morton_encode(ctx, coords))
    cmg.cmg_level_set_density(G, cfg["rho"][0], 1.0)
    rc, st_mg = cmg.cmg_level_solve(G, tol=1e-12)
    phi_mg = cmg.cmg_level_get_phi(G)
    cmg.cmg_level_set_phi(G, np.zeros_like(phi_mg))
    rc, st = cmg.cmg_level_solve(G, tol=1e-12, precision=cmg.CMG_PREC_FFT)
    assert st["rel_final"] <= 1e-12 and st["cycles"] <= 5
    phi = cmg.cmg_level_get_phi(G)
    assert relerr(phi, phi_mg) <= 1e-10
    R = O.Level(7, O.morton_encode(coords))
    R.set_density(cfg["rho"][0], 1.0)
    R.set_phi(phi)
    assert np.sqrt(R.residual(0, use_ghost=False)) <= 1.0001e-12 * st["norm0"]


def test_fft_rejects_levels_it_cannot_solve(cmg, ctx):
    cfg = inputs.two_level_amr(base_level=4, seed=2)
    B = cmg.cmg_level_build(ctx, 4, cmg.cmg_morton_encode(ctx, cfg["coords"][0]))
    F = cmg.cmg_level_build(ctx, 5, cmg.cmg_morton_encode(ctx, cfg["coords"][1]), parent=B)
    cmg.cmg_level_set_density(F, cfg["rho"][1], 1.0)
    with pytest.raises(cmg.CmgError) as e:
        cmg.cmg_level_solve(F, tol=1e-10, precision=cmg.CMG_PREC_FFT)
    assert e.value.code == cmg.CMG_ERR_INVALID_ARG
