"""The allocation-free residual norm (cmg_residual_norm2_noalloc).

It serves callers that cannot allocate device memory when they check a
residual: real-time loops that forbid allocation after start-up, hosts that
own all device memory in an arena of their own.  It must agree with the
library's own residual norm (cmg_level_mg_step with CMG_OP_RESIDUAL, which
reduces through scratch the level allocated), call after call, since every
call reuses the same static scratch array.

This file sorts last so that a stop-at-first-failure run has already run every
other test; it also passes on its own in a fresh process."""
import numpy as np
import pytest

from paper_2604_06035_gb300 import inputs

pytestmark = pytest.mark.gpu

RTOL_NORM = 1e-11  # the tolerance the other residual-norm tests use


@pytest.fixture(scope="module")
def cmg():
    import __graft_entry__ as ge
    ge.build()
    from paper_2604_06035_gb300 import cmg as _c
    return _c


def test_noalloc_norm_matches_library_norm_twice(cmg):
    import torch
    ctx = cmg.cmg_ctx_create(0)
    try:
        cfg = inputs.two_level_amr(base_level=5, seed=2)
        kb = cmg.cmg_morton_encode(ctx, cfg["coords"][0])
        kf = cmg.cmg_morton_encode(ctx, cfg["coords"][1])
        B = cmg.cmg_level_build(ctx, 5, kb)
        F = cmg.cmg_level_build(ctx, 6, kf, parent=B)
        rng = np.random.default_rng(31)
        cmg.cmg_level_set_phi(B, rng.standard_normal((cmg.cmg_level_n_octs(B), 8)))
        cmg.cmg_level_set_density(B, cfg["rho"][0], 1.0)
        cmg.cmg_level_set_phi(F, rng.standard_normal((cmg.cmg_level_n_octs(F), 8)))
        cmg.cmg_level_set_density(F, cfg["rho"][1], 1.0)
        cmg.cmg_level_mg_step(F, 0, cmg.CMG_OP_GHOSTS)
        stream = torch.cuda.current_stream()
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        # two calls in a row, on levels of different sizes: the fine level
        # (with coarse-fine ghosts) and then the periodic base level
        for L, h, with_ghosts in ((F, 1.0 / 64, True), (B, 1.0 / 32, False)):
            want = cmg.cmg_level_mg_step(L, 0, cmg.CMG_OP_RESIDUAL)
            nbr = cmg.cmg_level_get_neighbors(L, device=True)
            ghosts = cmg.cmg_level_get_ghosts(L, device=True) if with_ghosts else None
            phi = cmg.cmg_level_get_phi(L, device=True)
            f = cmg.cmg_level_mg_get(L, 0, cmg.CMG_FIELD_F, device=True)
            torch.cuda.synchronize()
            cmg.cmg_residual_norm2_noalloc(nbr, ghosts, phi, f, h, out, stream=stream)
            torch.cuda.synchronize()
            got = float(out.item())
            assert want > 0
            assert abs(got - want) <= RTOL_NORM * want, (got, want)
        with pytest.raises(cmg.CmgError):
            cmg.cmg_residual_norm2_noalloc(nbr, None, phi, f, -1.0, out, stream=stream)
        del F, B
    finally:
        import gc
        gc.collect()
        cmg.cmg_ctx_destroy(ctx)
