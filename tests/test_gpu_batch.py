"""Batched patch solve (one persistent cooperative kernel per solve) against
the CPU oracle solving each patch on its own.

With the V(2,2) schedule the coarsest solve of every patch is 4 red-black
sweeps, so a patch's result in the batch must equal the oracle's solve of
that patch alone with coarse_sweeps = 4: FP64 to 1e-12 relative at equal
cycle counts, the same cycle at which each patch reaches tol, and mixed
precision within 1e-10 of the FP64 solution.  With krylov = 1 each patch runs
the oracle's preconditioned CG of that patch alone."""
import numpy as np
import pytest

import oracle as O
from paper_2604_06035_gb300 import inputs

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
    cmg.cmg_ctx_destroy(c)


@pytest.fixture(scope="module")
def setup(cmg, ctx):
    b = inputs.batched_patches(n_patches=12, n_max=3000, seed=7)
    lev = b["level"]
    P = cmg.cmg_level_build(ctx, lev - 1, cmg.cmg_morton_encode(ctx, b["parent_coords"]))
    cmg.cmg_level_set_phi(P, b["parent_phi"])
    F = cmg.cmg_level_build(ctx, lev, cmg.cmg_morton_encode(ctx, b["coords"]), parent=P)
    cmg.cmg_level_set_density(F, b["rho"], 1.0)
    B = cmg.cmg_batch_create(F, b["offsets"])
    cmg.cmg_batch_set_schedule(B, threads=256, blocks_per_sm=2, n_pre=2, n_post=2, inner_cycles=1)
    RP = O.Level(lev - 1, O.morton_encode(b["parent_coords"]))
    RP.set_phi(b["parent_phi"])
    return b, P, F, B, RP


def _oracle_patch(b, RP, k):
    sl = slice(b["offsets"][k], b["offsets"][k + 1])
    R = O.Level(b["level"], O.morton_encode(b["coords"][sl]), parent=RP)
    R.set_density(b["rho"][sl], 1.0)
    return R, sl


def _relerr(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def test_batch_fp64_fixed_cycles_matches_per_patch_oracle(cmg, setup):
    b, P, F, B, RP = setup
    cmg.cmg_level_set_phi(F, np.zeros((len(b["coords"]), 8)))
    rc, st = cmg.cmg_batch_solve(B, tol=1e-10, fixed_cycles=3)
    assert rc == cmg.CMG_OK and st["cycles"] == 3 and st["grid_barriers"] > 0
    phi = cmg.cmg_level_get_phi(F)
    for k in range(len(b["offsets"]) - 1):
        R, sl = _oracle_patch(b, RP, k)
        R.solve(tol=1e-10, fixed_cycles=3, coarse_sweeps=4)
        assert _relerr(phi[sl], R.get_phi()) <= 1e-12, k


def test_batch_fp64_to_tolerance_per_patch_cycles(cmg, setup):
    b, P, F, B, RP = setup
    cmg.cmg_level_set_phi(F, np.zeros((len(b["coords"]), 8)))
    rc, st = cmg.cmg_batch_solve(B, tol=1e-10)
    assert rc == cmg.CMG_OK and st["n_converged"] == st["n_patches"] == 12
    rel, conv, n0 = cmg.cmg_batch_patch_stats(B)
    assert np.all(rel <= 1e-10) and np.all(conv >= 1) and st["cycles"] == conv.max()
    mismatched = 0
    for k in range(12):
        R, sl = _oracle_patch(b, RP, k)
        rc_o, so = R.solve(tol=1e-10, coarse_sweeps=4)
        mismatched += int(so["cycles"] != conv[k])
        assert abs(so["cycles"] - conv[k]) <= 1
        assert abs(n0[k] - so["norm0"]) <= 1e-12 * so["norm0"]
    assert mismatched <= 1


def test_batch_mixed_matches_fp64(cmg, setup):
    b, P, F, B, RP = setup
    cmg.cmg_level_set_phi(F, np.zeros((len(b["coords"]), 8)))
    rc, st = cmg.cmg_batch_solve(B, tol=1e-11, precision=cmg.CMG_PREC_MIXED)
    assert rc == cmg.CMG_OK and st["n_converged"] == 12
    phi = cmg.cmg_level_get_phi(F)
    for k in (0, 5, 11):
        R, sl = _oracle_patch(b, RP, k)
        R.solve(tol=1e-13, coarse_sweeps=4)
        assert _relerr(phi[sl], R.get_phi()) <= 1e-10, k


def test_batch_pcg_fixed_iterations_match_per_patch_oracle(cmg, setup):
    """krylov = 1: every patch runs its own flexible CG with the batch's
    V-cycle from zero as the preconditioner -- the oracle's PCG of the patch
    alone (coarsest = 4 sweeps).  Per-patch dot products are summed with
    atomics in the batch (a different order than the oracle's), which moves
    alpha and beta at the 1e-16 level: 1e-11 after three iterations."""
    b, P, F, B, RP = setup
    cmg.cmg_level_set_phi(F, np.zeros((len(b["coords"]), 8)))
    rc, st = cmg.cmg_batch_solve(B, tol=1e-10, fixed_cycles=3, krylov=1)
    assert rc == cmg.CMG_OK and st["cycles"] == 3
    phi = cmg.cmg_level_get_phi(F)
    for k in range(len(b["offsets"]) - 1):
        R, sl = _oracle_patch(b, RP, k)
        R.solve_pcg(tol=1e-10, fixed_cycles=3, coarse_sweeps=4)
        assert _relerr(phi[sl], R.get_phi()) <= 1e-11, k


def test_batch_pcg_to_tolerance(cmg, setup):
    b, P, F, B, RP = setup
    z = np.zeros((len(b["coords"]), 8))
    cmg.cmg_level_set_phi(F, z)
    rc, st_mg = cmg.cmg_batch_solve(B, tol=1e-10)
    cmg.cmg_level_set_phi(F, z)
    rc, st = cmg.cmg_batch_solve(B, tol=1e-10, krylov=1)
    assert rc == cmg.CMG_OK and st["n_converged"] == 12
    assert st["cycles"] < st_mg["cycles"]
    rel, conv, n0 = cmg.cmg_batch_patch_stats(B)
    assert np.all(rel <= 1e-10) and st["cycles"] == conv.max()
    phi = cmg.cmg_level_get_phi(F)
    for k in range(12):
        R, sl = _oracle_patch(b, RP, k)
        rc_o, so = R.solve_pcg(tol=1e-10, coarse_sweeps=4)
        assert abs(so["cycles"] - conv[k]) <= 1, k
        R.solve(tol=1e-13, coarse_sweeps=4)
        assert _relerr(phi[sl], R.get_phi()) <= 1e-8, k
    # the level is left as a solve leaves it (source restored, ghosts refilled):
    # a stationary solve from this phi has nothing to do
    rc, st2 = cmg.cmg_batch_solve(B, tol=1e-10)
    assert rc == cmg.CMG_OK and st2["cycles"] == 0


def test_batch_pcg_mixed_matches_fp64(cmg, setup):
    b, P, F, B, RP = setup
    z = np.zeros((len(b["coords"]), 8))
    cmg.cmg_level_set_phi(F, z)
    rc, st_mg = cmg.cmg_batch_solve(B, tol=1e-11, precision=cmg.CMG_PREC_MIXED)
    cmg.cmg_level_set_phi(F, z)
    rc, st = cmg.cmg_batch_solve(B, tol=1e-11, precision=cmg.CMG_PREC_MIXED, krylov=1)
    assert rc == cmg.CMG_OK and st["n_converged"] == 12
    assert st["cycles"] <= st_mg["cycles"]
    phi = cmg.cmg_level_get_phi(F)
    for k in (0, 5, 11):
        R, sl = _oracle_patch(b, RP, k)
        R.solve(tol=1e-13, coarse_sweeps=4)
        assert _relerr(phi[sl], R.get_phi()) <= 1e-10, k


def test_batch_cg_allocation_failure_then_success(cmg, setup):
    """The CG buffers of a batch are allocated on first use: an injected
    allocation failure there returns CMG_ERR_OOM, and the next solve
    allocates them and converges."""
    b, P, F, B, RP = setup
    z = np.zeros((len(b["coords"]), 8))
    B2 = cmg.cmg_batch_create(F, b["offsets"])
    try:
        for after in (1, 2):
            cmg.cmg_level_set_phi(F, z)
            cmg.cmg_debug_inject_alloc_failure(after)
            rc, st = cmg.cmg_batch_solve(B2, tol=1e-10, krylov=1, raise_on_error=False)
            cmg.cmg_debug_inject_alloc_failure(0)
            assert rc == cmg.CMG_ERR_OOM, after
        cmg.cmg_level_set_phi(F, z)
        rc, st = cmg.cmg_batch_solve(B2, tol=1e-10, krylov=1)
        assert rc == cmg.CMG_OK and st["n_converged"] == 12
    finally:
        cmg.cmg_debug_inject_alloc_failure(0)
        cmg.cmg_batch_destroy(B2)


def test_batch_rejects_patches_that_touch(cmg, setup):
    b, P, F, B, RP = setup
    off = b["offsets"]
    # split patch 0 into two ranges: its two halves are neighbours
    bad = np.concatenate([[0, off[1] // 2], off[1:]])
    with pytest.raises(cmg.CmgError) as e:
        cmg.cmg_batch_create(F, bad)
    assert e.value.code == cmg.CMG_ERR_INVALID_ARG


def test_batch_barrier_timeout_returns_status(cmg, setup):
    """A grid barrier that runs out of spin budget ends the persistent kernel
    with CMG_ERR_TIMEOUT; the context stays usable."""
    b, P, F, B, RP = setup
    cmg.cmg_batch_set_spin_budget(B, 0)
    rc, st = cmg.cmg_batch_solve(B, tol=1e-10, raise_on_error=False)
    assert rc == cmg.CMG_ERR_TIMEOUT
    cmg.cmg_batch_set_spin_budget(B, 2_000_000_000)
    cmg.cmg_level_set_phi(F, np.zeros((len(b["coords"]), 8)))
    rc, st = cmg.cmg_batch_solve(B, tol=1e-10)
    assert rc == cmg.CMG_OK and st["n_converged"] == 12


def test_batch_autotune(cmg, setup):
    b, P, F, B, RP = setup
    cmg.cmg_level_set_phi(F, np.zeros((len(b["coords"]), 8)))
    before = cmg.cmg_level_get_phi(F)
    best, ms = cmg.cmg_batch_autotune(B, tol=1e-10, precision=cmg.CMG_PREC_MIXED)
    assert np.array_equal(cmg.cmg_level_get_phi(F), before)
    assert best["threads"] in (256, 512) and best["n_pre"] >= 1 and ms > 0
    assert cmg.cmg_batch_get_schedule(B) == best
    rc, st = cmg.cmg_batch_solve(B, tol=1e-10, precision=cmg.CMG_PREC_MIXED)
    assert rc == cmg.CMG_OK and st["n_converged"] == 12
    cmg.cmg_batch_set_schedule(B, threads=256, blocks_per_sm=2, n_pre=2, n_post=2, inner_cycles=1)


def test_full_batch_sampled_patches_match_oracle(cmg, ctx):
    """The benchmark's batch (512 patches, 14.7 M octs) in the launch shape
    its FP64 autotuning picks (512 threads, one block per SM, V(2,3)): two
    FP64 V-cycles of the whole batch, then 13 patches sampled across the size
    range, each against the oracle solving that patch alone with the same
    schedule and coarse_sweeps = n_pre + n_post = 5 (1e-12)."""
    import os
    b = inputs.batched_patches(n_patches=512, seed=4)
    lev = b["level"]
    P = cmg.cmg_level_build(ctx, lev - 1, cmg.cmg_morton_encode(ctx, b["parent_coords"]))
    cmg.cmg_level_set_phi(P, b["parent_phi"])
    F = cmg.cmg_level_build(ctx, lev, cmg.cmg_morton_encode(ctx, b["coords"]), parent=P)
    cmg.cmg_level_set_density(F, b["rho"], 1.0)
    B = cmg.cmg_batch_create(F, b["offsets"])
    cmg.cmg_batch_set_schedule(B, threads=512, blocks_per_sm=1, n_pre=2, n_post=3, inner_cycles=1)
    cmg.cmg_level_set_phi(F, np.zeros((len(b["coords"]), 8)))
    rc, st = cmg.cmg_batch_solve(B, tol=1e-10, fixed_cycles=2)
    assert rc == cmg.CMG_OK and st["cycles"] == 2
    phi = cmg.cmg_level_get_phi(F)
    cmg.cmg_batch_destroy(B)
    cmg.cmg_level_destroy(F)
    cmg.cmg_level_destroy(P)
    sizes = np.diff(b["offsets"])
    order = np.argsort(sizes)
    sample = order[np.linspace(0, len(order) - 1, 13).round().astype(int)]
    threads = O.get_threads()
    O.set_threads(len(os.sched_getaffinity(0)))
    try:
        RP = O.Level(lev - 1, O.morton_encode(b["parent_coords"]))
        RP.set_phi(b["parent_phi"])
        for k in sample:
            R, sl = _oracle_patch(b, RP, int(k))
            R.solve(tol=1e-10, fixed_cycles=2, n_pre=2, n_post=3, coarse_sweeps=5)
            assert _relerr(phi[sl], R.get_phi()) <= 1e-12, (int(k), int(sizes[k]))
    finally:
        O.set_threads(threads)
