"""The oracle's 128-bit Morton keys (Sec. 4.2, B = 42 bits per coordinate,
levels up to 43) and the level build on them, pinned against independent
arithmetic: Python's unbounded integers for the bit interleave, dictionaries
for the hash lookups, coordinate arithmetic for the neighbours, and the 64-bit
build, which the 128-bit one must reproduce wherever coordinates fit 21 bits."""
import numpy as np
import pytest

import oracle as O
from paper_2604_06035_gb300 import inputs


def _interleave(i, j, k, bits=42):
    m = 0
    for b in range(bits):
        m |= ((i >> b) & 1) << (3 * b) | ((j >> b) & 1) << (3 * b + 1) | ((k >> b) & 1) << (3 * b + 2)
    return m


def _words(m):
    return m & ((1 << 64) - 1), m >> 64


def test_morton128_bit_layout_and_round_trip():
    rng = np.random.default_rng(1)
    ijk = rng.integers(0, 1 << 42, size=(500, 3), dtype=np.uint64)
    ijk[:8] = [[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [(1 << 21) - 1] * 3, [1 << 21] * 3,
               [(1 << 42) - 1] * 3, [(1 << 21) + 1, 3, (1 << 41)]]
    keys = O.morton_encode128(ijk)
    for t in range(len(ijk)):
        m = _interleave(*(int(v) for v in ijk[t]))
        assert (int(keys[t, 0]), int(keys[t, 1])) == _words(m)
    assert np.array_equal(O.morton_decode128(keys), ijk)
    # below 2^21 per coordinate the 128-bit key is the 64-bit key
    small = ijk[:, :] % (1 << 21)
    k128 = O.morton_encode128(small)
    assert np.array_equal(k128[:, 0], O.morton_encode(small.astype(np.uint32))) and not k128[:, 1].any()
    # the parent oct (key >> 3) holds the halved coordinates
    for t in range(50):
        m = int(keys[t, 0]) | int(keys[t, 1]) << 64
        pw = np.array([_words(m >> 3)], dtype=np.uint64)
        assert np.array_equal(O.morton_decode128(pw)[0], ijk[t] >> 1)


def _build_chain(cfg):
    R = []
    for lev, c in zip(cfg["levels"], cfg["coords"]):
        R.append(O.Level(lev, O.morton_encode128(c), parent=R[-1] if R else None))
    return R


def test_deep_zoom_lookups_neighbours_and_fathers_by_brute_force():
    cfg = inputs.deep_zoom(top_level=30)
    R = _build_chain(cfg)
    for lev, c, L in list(zip(cfg["levels"], cfg["coords"], R))[-3:]:
        assert lev > 22 and L.wide
        pos = {tuple(int(v) for v in x): t for t, x in enumerate(c)}
        keys = O.morton_encode128(c)
        assert np.array_equal(L.lookup(keys), np.arange(len(c)))
        # absent keys: shifted outside the cube
        q = O.morton_encode128(c + np.uint64(1 << 20))
        assert np.all(L.lookup(q) == -1)
        nb = L.neighbors()
        for t, x in enumerate(c):
            for d in range(6):
                y = [int(v) for v in x]
                y[d // 2] += 1 if d & 1 else -1
                assert nb[t, 1 + d] == pos.get(tuple(y), -1)
        # father cells of missing neighbours: the parent oct of the neighbour
        # position and its octant
        par = {tuple(int(v) for v in x): t for t, x in enumerate(cfg["coords"][cfg["levels"].index(lev) - 1])}
        fc = L.father_cells()
        for t, x in enumerate(c[:64]):
            for d in range(6):
                if nb[t, 1 + d] >= 0:
                    continue
                y = [int(v) for v in x]
                y[d // 2] += 1 if d & 1 else -1
                oc = (y[0] & 1) | (y[1] & 1) << 1 | (y[2] & 1) << 2
                assert tuple(fc[t, d]) == (par[tuple(v >> 1 for v in y)], oc)


def test_128bit_build_reproduces_64bit_build():
    """Coordinates below 2^21: the 128-bit keys' hash (XOR fold, App. B) is the
    64-bit key's, so neighbours, father cells, hierarchy and a solve agree
    exactly."""
    cfg = inputs.two_level_amr(base_level=5, seed=2)
    A, W = [], []
    for lev, c in zip(cfg["levels"], cfg["coords"]):
        A.append(O.Level(lev, O.morton_encode(c), parent=A[-1] if A else None))
        W.append(O.Level(lev, O.morton_encode128(c.astype(np.uint64)), parent=W[-1] if W else None))
    for a, w, rho in zip(A, W, cfg["rho"]):
        assert a.hash_capacity == w.hash_capacity
        assert np.array_equal(a.neighbors(), w.neighbors())
        assert np.array_equal(a.father_cells(), w.father_cells())
        assert a.mg_depth == w.mg_depth
        for m in range(a.mg_depth):
            assert np.array_equal(a.mg_keys(m), w.mg_keys(m)[:, 0]) and not w.mg_keys(m)[:, 1].any()
        a.set_density(rho, 1.0)
        w.set_density(rho, 1.0)
        a.solve(fixed_cycles=3)
        w.solve(fixed_cycles=3)
        assert np.array_equal(a.get_phi(), w.get_phi())


def test_deep_zoom_chain_solves_to_tolerance():
    cfg = inputs.deep_zoom(top_level=26)
    R = _build_chain(cfg)
    for k, (L, rho) in enumerate(zip(R, cfg["rho"])):
        L.set_density(rho, cfg["rho_bar"])
        rc, st = L.solve(tol=1e-10)
        assert st["rel_final"] <= 1e-10, k
        assert np.sqrt(L.residual(0, use_ghost=k > 0)) <= 1.0001e-10 * st["norm0"], k


def test_wide_key_errors():
    c = np.array([[0, 0, 0]], dtype=np.uint64)
    with pytest.raises(O.OracleError):
        O.Level(44, O.morton_encode128(c), periodic_mask=0)  # beyond B = 42
    with pytest.raises(O.OracleError):
        O.Level(23, O.morton_encode(c.astype(np.uint32)), periodic_mask=0)  # 64-bit keys stop at 22
    bad = O.morton_encode128(np.array([[1 << 30, 0, 0]], dtype=np.uint64))
    with pytest.raises(O.OracleError):
        O.Level(30, bad, periodic_mask=0)  # coordinate >= 2^29 at level 30
