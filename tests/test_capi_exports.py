"""CPU-side checks of the C-ABI boundary: libcmg.so builds for sm_103a, loads
without a GPU, and exports every function include/cmg.h declares; the binding
covers exactly those names; product code never reaches the oracle."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "cmg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(cmg_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2604_06035_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["cmg_ctx_create", "cmg_level_build", "cmg_level_set_density", "cmg_level_solve",
                 "cmg_level_get_phi", "cmg_level_get_residual", "cmg_level_lookup", "cmg_morton_encode"]:
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_matches_header(libpath):
    from paper_2604_06035_gb300 import cmg
    assert set(cmg.exported_symbols()) == set(declared_functions())
    for n in declared_functions():
        assert hasattr(cmg, n), n
    assert cmg.cmg_version().startswith("cmg ")


def test_context_without_gpu_fails_loudly(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2604_06035_gb300 import cmg
    with pytest.raises(cmg.CmgError) as e:
        cmg.cmg_ctx_create(0, stream=0)
    assert e.value.code in (cmg.CMG_ERR_CUDA, cmg.CMG_ERR_INVALID_ARG)


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2604_06035_gb300")
    bad = re.compile(r"^\s*(import\s+oracle|from\s+oracle|#\s*include\s*[<\"].*oracle)|liboracle", re.M)
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                assert not bad.search(open(os.path.join(dirpath, f)).read()), f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".c", ".h", ".py")):
            text = open(os.path.join(ROOT, "oracle", f)).read()
            assert "paper_2604_06035_gb300" not in text and "cmg_internal" not in text, f


def test_noalloc_rejects_sizes_beyond_its_scratch(libpath):
    """The size check comes before any CUDA call, so this runs without a GPU:
    2^24 + 1 octs would need more block sums than the static scratch holds."""
    from paper_2604_06035_gb300 import cmg
    lib = cmg.lib()
    dummy = ctypes.c_void_p(0x1000)
    rc = lib.cmg_residual_norm2_noalloc(dummy, None, dummy, dummy, (1 << 24) + 1, 1.0, dummy, ctypes.c_void_p(0))
    assert rc == cmg.CMG_ERR_INVALID_ARG
    rc = lib.cmg_residual_norm2_noalloc(dummy, None, dummy, dummy, 8, -1.0, dummy, ctypes.c_void_p(0))
    assert rc == cmg.CMG_ERR_INVALID_ARG


def test_noalloc_binding_checks_array_sizes(libpath):
    """The binding rejects arrays shorter (or longer) than the n octs the
    neighbour table implies before it reaches the library."""
    import numpy as np
    from paper_2604_06035_gb300 import cmg
    n = 16
    nbr = np.zeros((n, 7), dtype=np.int32)
    good = np.zeros((n, 8))
    out = np.zeros(1)
    cases = [
        (nbr, None, good[:-1], good, out),          # phi short by one oct
        (nbr, None, good, good[:, :6], out),        # f with 6 values per oct
        (nbr, np.zeros((n, 6)), good, good, out),   # ghosts [n][6] instead of [n][6][4]
        (nbr[:, :6], None, good, good, out),        # neighbours [n][6]
        (nbr, None, good, good, np.zeros(0)),       # no room for the result
    ]
    for neighbors, ghosts, phi, f, norm2 in cases:
        with pytest.raises(ValueError):
            cmg.cmg_residual_norm2_noalloc(neighbors, ghosts, phi, f, 1.0, norm2)
