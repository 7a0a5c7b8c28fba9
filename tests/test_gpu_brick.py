"""The shared-memory brick kernel for the colour passes of lexicographic full
periodic levels (brick.cu): it must give the neighbour-table kernel's bits
(same operands, same order, same sum), in FP64 and FP32, on every MG level it
runs on, and must not run on a full periodic level whose octs are not in
lexicographic order (its implicit neighbours would be wrong there)."""
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
    import gc
    gc.collect()
    cmg.cmg_ctx_destroy(c)


def _solve(cmg, L, rho, staged, prec, cycles):
    cmg.cmg_level_set_stencil(L, staged)
    cmg.cmg_level_set_density(L, rho, 1.0)
    cmg.cmg_level_set_phi(L, np.zeros_like(rho))
    cmg.cmg_level_solve(L, fixed_cycles=cycles, precision=prec)
    return cmg.cmg_level_get_phi(L)


@pytest.mark.parametrize("level,tails", [(6, (0, 0)), (7, (-1, -1))])
def test_brick_matches_table_kernel_bit_for_bit(cmg, ctx, level, tails):
    coords = inputs.uniform_oct_coords(level)
    rho = 1.0 + inputs.grf(1 << level, 0.5, seed=3).astype(np.float64)
    rho = inputs.dense_to_octs(rho, coords)
    L = cmg.cmg_level_build(ctx, level, cmg.cmg_morton_encode(ctx, coords))
    cmg.cmg_level_set_schedule(L, *tails)  # (0, 0): every MG level in per-operation kernels
    for prec in (cmg.CMG_PREC_FP64, cmg.CMG_PREC_MIXED):
        a = _solve(cmg, L, rho, 2, prec, 3)  # brick kernel for FP32 and FP64 passes
        b = _solve(cmg, L, rho, 0, prec, 3)  # neighbour-table kernel
        c = _solve(cmg, L, rho, 1, prec, 3)  # the default split
        assert np.array_equal(a.view(np.uint64), b.view(np.uint64)), prec
        assert np.array_equal(c.view(np.uint64), b.view(np.uint64)), prec
    # and the oracle, FP64 at equal cycles
    ol = O.Level(level, O.morton_encode(coords))
    ol.set_density(rho, 1.0)
    ol.solve(fixed_cycles=3)
    want = ol.get_phi()
    got = _solve(cmg, L, rho, 2, cmg.CMG_PREC_FP64, 3)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


def test_shuffled_full_level_is_not_taken_for_lexicographic(cmg, ctx):
    level = 6
    coords = inputs.uniform_oct_coords(level)
    perm = np.random.default_rng(9).permutation(len(coords))
    # one swap of two octs is enough to break the implicit neighbours
    swap = np.arange(len(coords))
    swap[[5, 700]] = swap[[700, 5]]
    rho = inputs.dense_to_octs(1.0 + inputs.grf(1 << level, 0.5, seed=4).astype(np.float64), coords)
    for order in (perm, swap):
        c = coords[order]
        L = cmg.cmg_level_build(ctx, level, cmg.cmg_morton_encode(ctx, c))
        cmg.cmg_level_set_schedule(L, 0, 0)
        got = _solve(cmg, L, rho[order], 2, cmg.CMG_PREC_FP64, 2)
        ol = O.Level(level, O.morton_encode(c))
        ol.set_density(rho[order], 1.0)
        ol.solve(fixed_cycles=2)
        want = ol.get_phi()
        assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))
        del L


def test_stencil_switch_rejects_bad_values(cmg, ctx):
    L = cmg.cmg_level_build(ctx, 5, cmg.cmg_morton_encode(ctx, inputs.uniform_oct_coords(5)))
    with pytest.raises(cmg.CmgError):
        cmg.cmg_level_set_stencil(L, 3)
    with pytest.raises(cmg.CmgError):
        cmg.cmg_level_set_stencil(L, -1)
