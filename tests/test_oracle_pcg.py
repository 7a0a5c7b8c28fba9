"""Pins of the oracle's multigrid-preconditioned conjugate gradients (the
paper names multigrid as the CG preconditioner, App. D.2): its solution is
the exact discrete solution (closed form by FFT on periodic levels) and the
solution the stationary V-cycle reaches; a near-exact preconditioner makes
CG finish in one or two iterations; and CG needs fewer V-cycles than the
stationary iteration."""
import numpy as np

import oracle as O
from paper_2604_06035_gb300 import inputs
from tests import dense_ref as D


def test_pcg_periodic_matches_exact_fft_solution():
    level = 4
    cfg = inputs.periodic_grf_level(level, rms=0.5, seed=7)
    coords = cfg["coords"][0]
    R = O.Level(level, O.morton_encode(coords))
    R.set_density(cfg["rho"][0], 1.0)
    rc, st = R.solve_pcg(tol=1e-13)
    n = 1 << level
    f = inputs.octs_to_dense(cfg["rho"][0] - 1.0, coords, n)
    exact = inputs.dense_to_octs(D.fft_solve(f, 1.0 / n), coords)
    phi = R.get_phi()
    assert np.max(np.abs(phi - exact)) <= 1e-11 * np.max(np.abs(exact))
    assert st["rel_final"] <= 1e-13


def test_pcg_refined_level_matches_stationary_multigrid():
    cfg = inputs.two_level_amr(base_level=5, seed=2)
    B = O.Level(5, O.morton_encode(cfg["coords"][0]))
    F = O.Level(6, O.morton_encode(cfg["coords"][1]), parent=B)
    B.set_density(cfg["rho"][0], 1.0)
    F.set_density(cfg["rho"][1], 1.0)
    B.solve(tol=1e-13)
    rc, s_mg = F.solve(tol=1e-13)
    a = F.get_phi()
    F.set_phi(np.zeros_like(a))
    rc, s_cg = F.solve_pcg(tol=1e-13)
    b = F.get_phi()
    assert np.max(np.abs(a - b)) <= 1e-11 * np.max(np.abs(a))
    assert s_cg["cycles"] < s_mg["cycles"]
    # the CG recurrence residual tracks the true residual
    n2 = F.residual(0, use_ghost=True)
    assert np.sqrt(n2) <= 2e-13 * s_cg["norm0"]


def test_pcg_with_near_exact_preconditioner_finishes_at_once():
    """With V(30, 30) cycles and 200 coarsest sweeps on a small refined level
    the preconditioner is close to the exact inverse: CG stops after one or
    two iterations, where the plain V(2, 2) preconditioner needs more."""
    cfg = inputs.two_level_amr(base_level=3, seed=2)
    B = O.Level(3, O.morton_encode(cfg["coords"][0]))
    F = O.Level(4, O.morton_encode(cfg["coords"][1]), parent=B)
    B.set_density(cfg["rho"][0], 1.0)
    F.set_density(cfg["rho"][1], 1.0)
    B.solve(tol=1e-13)
    rc, st = F.solve_pcg(tol=1e-8, n_pre=30, n_post=30, coarse_sweeps=200)
    assert st["cycles"] <= 2 and st["rel_final"] <= 1e-8
    F.set_phi(np.zeros((F.n, 8)))
    rc, st2 = F.solve_pcg(tol=1e-8)
    assert st2["cycles"] > st["cycles"]


def test_pcg_fixed_iterations_and_zero_source():
    cfg = inputs.periodic_grf_level(4, rms=0.5, seed=2)
    R = O.Level(4, O.morton_encode(cfg["coords"][0]))
    R.set_density(np.ones_like(cfg["rho"][0]), 1.0)  # f = 0
    rc, st = R.solve_pcg(tol=1e-10)
    assert np.all(R.get_phi() == 0.0) and st["cycles"] == 0
    R.set_density(cfg["rho"][0], 1.0)
    R.set_phi(np.zeros((R.n, 8)))
    rc, st = R.solve_pcg(fixed_cycles=3)
    assert st["cycles"] == 3 and len(st["rel_history"]) == 3
    assert st["rel_history"][2] < st["rel_history"][0]
