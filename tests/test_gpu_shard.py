"""The sharded level solve on the GPU through the C ABI (range operations and
cell gather / scatter of libcmg.so), two ranks as threads of one process, each
with its own context and replica of the level; exchanges go through the host
between operations, so no kernel of one rank waits on another's.

Against the single-rank GPU solve with the same oct order: bit for bit on a
refined level with a given parent phi, to rounding on the periodic base (its
mean is removed from all-reduced sums).  Against the oracle: 1e-12."""
import threading

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


def _run_ranks(cmg, world, make_level, cycles):
    """make_level(ctx) -> (level handle, refined).  Returns per-rank
    (lo, hi, phi rows, stats)."""
    from paper_2604_06035_gb300 import shard as S
    hub = S.LocalHub(world)
    res, err = [None] * world, []

    def run(r):
        ctx = cmg.cmg_ctx_create(0)
        try:
            L, refined = make_level(ctx)
            be = S.CmgBackend(L, refined=refined)
            keys, act, levs = be.hierarchy()
            owner0 = S.ksection(S.morton_decode(keys[0]), world)
            plan = S.ShardPlan.build(keys, act, levs, owner0, world)
            st = S.ShardedSolver(be, plan, hub.comm(r)).solve(fixed_cycles=cycles)
            lo, hi = plan.ranges[0][r]
            res[r] = (lo, hi, cmg.cmg_level_get_phi(L)[lo:hi], st)
            del L
        except Exception as e:  # surfaced by the caller
            err.append(e)
            hub.barrier.abort()
        finally:
            import gc
            gc.collect()
            cmg.cmg_ctx_destroy(ctx)

    ts = [threading.Thread(target=run, args=(r,)) for r in range(world)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not err, err
    return res


def _sorted(coords, world):
    from paper_2604_06035_gb300 import shard as S
    return S.owner_order(S.ksection(coords, world))


def test_two_rank_refined_level_is_bit_identical(cmg):
    world, cycles = 2, 3
    cfg = inputs.two_level_amr(base_level=6, seed=2)
    perm = _sorted(cfg["coords"][1], world)
    pphi = np.random.default_rng(11).standard_normal((len(cfg["coords"][0]), 8))

    def make(ctx):
        B = cmg.cmg_level_build(ctx, 6, cmg.cmg_morton_encode(ctx, cfg["coords"][0]))
        cmg.cmg_level_set_phi(B, pphi)
        F = cmg.cmg_level_build(ctx, 7, cmg.cmg_morton_encode(ctx, cfg["coords"][1][perm]), parent=B)
        cmg.cmg_level_set_density(F, cfg["rho"][1][perm], 1.0)
        cmg.cmg_level_set_phi(F, np.zeros((len(perm), 8)))
        return F, True

    res = _run_ranks(cmg, world, make, cycles)
    got = np.zeros((len(perm), 8))
    for lo, hi, phi, st in res:
        got[lo:hi] = phi
        assert st["exchanges"] > 0 and st["cycles"] == cycles
    # the single-rank GPU solve of the same level
    ctx = cmg.cmg_ctx_create(0)
    try:
        F, _ = make(ctx)
        cmg.cmg_level_solve(F, fixed_cycles=cycles)
        ref = cmg.cmg_level_get_phi(F)
        del F
    finally:
        import gc
        gc.collect()
        cmg.cmg_ctx_destroy(ctx)
    assert np.array_equal(got, ref)
    # and the oracle with the same parent phi
    ob = O.Level(6, O.morton_encode(cfg["coords"][0]))
    ob.set_phi(pphi)
    of = O.Level(7, O.morton_encode(cfg["coords"][1][perm]), parent=ob)
    of.set_density(cfg["rho"][1][perm], 1.0)
    of.solve(fixed_cycles=cycles)
    want = of.get_phi()
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


def test_two_rank_periodic_level_matches(cmg):
    world, cycles = 2, 4
    cfg = inputs.two_level_amr(base_level=6, seed=2)
    perm = _sorted(cfg["coords"][0], world)

    def make(ctx):
        B = cmg.cmg_level_build(ctx, 6, cmg.cmg_morton_encode(ctx, cfg["coords"][0][perm]))
        cmg.cmg_level_set_density(B, cfg["rho"][0][perm], 1.0)
        cmg.cmg_level_set_phi(B, np.zeros((len(perm), 8)))
        return B, False

    res = _run_ranks(cmg, world, make, cycles)
    got = np.zeros((len(perm), 8))
    for lo, hi, phi, st in res:
        got[lo:hi] = phi
    ctx = cmg.cmg_ctx_create(0)
    try:
        B, _ = make(ctx)
        cmg.cmg_level_solve(B, fixed_cycles=cycles)
        ref = cmg.cmg_level_get_phi(B)
        del B
    finally:
        import gc
        gc.collect()
        cmg.cmg_ctx_destroy(ctx)
    assert np.max(np.abs(got - ref)) <= 1e-14 * np.max(np.abs(ref))
    ob = O.Level(6, O.morton_encode(cfg["coords"][0][perm]))
    ob.set_density(cfg["rho"][0][perm], 1.0)
    ob.solve(fixed_cycles=cycles)
    want = ob.get_phi()
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))
    # every rank ends with the same all-reduced residual history
    assert len({tuple(r[3]["rel_history"]) for r in res}) == 1


def test_range_and_cell_calls_reject_bad_arguments(cmg):
    import torch
    ctx = cmg.cmg_ctx_create(0)
    try:
        coords = inputs.uniform_oct_coords(3)
        L = cmg.cmg_level_build(ctx, 3, cmg.cmg_morton_encode(ctx, coords))
        n = cmg.cmg_level_n_octs(L)
        with pytest.raises(cmg.CmgError):
            cmg.cmg_level_mg_step_range(L, 0, cmg.CMG_OPR_SWEEP, 0, 0, n + 1)
        with pytest.raises(cmg.CmgError):
            cmg.cmg_level_mg_step_range(L, 0, cmg.CMG_OPR_SWEEP, 4, 0, n)
        cells = torch.tensor([0, 8 * n], dtype=torch.int32, device="cuda")
        with pytest.raises(cmg.CmgError):
            cmg.cmg_level_mg_gather(L, 0, 0, cells)
        # the context still works after the rejected index
        ok = torch.tensor([0, 8 * n - 1], dtype=torch.int32, device="cuda")
        v = cmg.cmg_level_mg_gather(L, 0, 0, ok)
        assert v.shape == (2,)
        del L
    finally:
        import gc
        gc.collect()
        cmg.cmg_ctx_destroy(ctx)
