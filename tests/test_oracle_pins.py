"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: hand-worked
keys from Eq. (morton_encode), brute-force searches, Python dicts, independent
dense-array operators, exact discrete and continuum solutions, and invariants.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from paper_2604_06035_gb300 import inputs
from tests import dense_ref as D

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def keys_of(coords):
    return O.morton_encode(np.asarray(coords, dtype=np.uint32))


# ------------------------------------------------------------------ Morton

def test_morton_hand_values():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "morton_hand.txt")) if l.strip() and l[0] != "#"]
    ijk = np.array([[int(r[0]), int(r[1]), int(r[2])] for r in rows], dtype=np.uint32)
    want = np.array([int(r[3]) for r in rows], dtype=np.uint64)
    assert np.array_equal(O.morton_encode(ijk), want)
    assert np.array_equal(O.morton_decode(want), ijk)


def test_morton_roundtrip_and_range():
    rng = np.random.default_rng(0)
    ijk = rng.integers(0, 1 << 21, size=(20000, 3), dtype=np.uint32)
    k = O.morton_encode(ijk)
    assert np.all(k < np.uint64(1 << 63))
    assert np.array_equal(O.morton_decode(k), ijk)
    # keys are a bijection: distinct coordinates give distinct keys
    u = np.unique(ijk, axis=0)
    assert len(np.unique(O.morton_encode(u))) == len(u)


def test_morton_parent_child():
    rng = np.random.default_rng(1)
    ijk = rng.integers(0, 1 << 20, size=(5000, 3), dtype=np.uint32)
    k = O.morton_encode(ijk)
    assert np.array_equal(O.morton_encode(ijk >> 1), k >> np.uint64(3))
    for c in range(8):
        b = np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1], dtype=np.uint32)
        kc = O.morton_encode(2 * ijk + b)
        assert np.array_equal(kc, (k << np.uint64(3)) | np.uint64(c))


def _z_order(n):
    """Recursive octant traversal (child c = bx + 2 by + 4 bz) of an n^3 grid."""
    if n == 1:
        return [(0, 0, 0)]
    sub = _z_order(n // 2)
    out = []
    for s in sub:
        for c in range(8):
            out.append((2 * s[0] + (c & 1), 2 * s[1] + ((c >> 1) & 1), 2 * s[2] + ((c >> 2) & 1)))
    return out


def test_morton_order_is_recursive_z_order():
    order = np.array(_z_order(8), dtype=np.uint32)
    k = O.morton_encode(order)
    assert np.array_equal(k, np.arange(512, dtype=np.uint64))


@pytest.mark.parametrize("level,nx", [(22, 1), (20, 4), (4, 1)])
def test_neighbor_walk_periodic(level, nx):
    npd = nx << (level - 1)
    assert npd <= 1 << 21
    rng = np.random.default_rng(level)
    for _ in range(20):
        ijk = rng.integers(0, npd, size=3).astype(np.uint32)
        m = int(keys_of([ijk])[0])
        for d in range(6):
            back = O.neighbor_key(O.neighbor_key(m, d, npd), d ^ 1, npd)
            assert back == m
            nk = O.neighbor_key(m, d, npd)
            got = O.morton_decode([nk])[0].astype(np.int64)
            want = ijk.astype(np.int64)
            want[d // 2] = (want[d // 2] + (1 if d & 1 else -1)) % npd
            assert np.array_equal(got, want)
    # a full walk along +x around the box comes back (small box only)
    if npd <= 16:
        m0 = m
        for _ in range(npd):
            m = O.neighbor_key(m, 1, npd)
        assert m == m0
    # the top corner wraps to zero on a periodic box and leaves a closed one
    top = int(keys_of([[npd - 1, npd - 1, npd - 1]])[0])
    assert O.neighbor_key(top, 1, npd, 7) == int(keys_of([[0, npd - 1, npd - 1]])[0])
    assert O.neighbor_key(top, 1, npd, 0) == -1
    assert O.neighbor_key(0, 0, npd, 0) == -1


# -------------------------------------------------------------------- hash

def test_hash_constants_and_semantics():
    g = json.load(open(os.path.join(GOLDEN, "paper_constants.json")))
    p1 = g["hash_phi1"]["value"]
    p2 = int(g["hash_phi2"]["value"], 16)
    M64 = (1 << 64) - 1
    rng = np.random.default_rng(2)
    for h in [0, 1, 2, 7, 1 << 62, (1 << 63) - 1] + [int(x) for x in rng.integers(0, 1 << 62, 50)]:
        t = (((h * p1) & M64) ^ (h >> 16)) * p2 & M64
        assert O.hash_fn(h) == (t ^ (t >> 13))


@pytest.mark.parametrize("n", [0, 1, 5, 7, 8, 1000, 4096])
def test_hash_capacity_rule(n):
    cap = O.hash_capacity_for(n)
    assert cap & (cap - 1) == 0
    assert n <= 0.7 * cap
    assert cap == 1 or n > 0.7 * (cap // 2)


@pytest.mark.parametrize("dense", [True, False])
def test_hash_lookup_vs_dict(dense):
    rng = np.random.default_rng(3)
    npd = 16 if dense else 1 << 20
    coords = rng.integers(0, npd, size=(3000, 3), dtype=np.uint32)
    coords = np.unique(coords, axis=0)
    rng.shuffle(coords)
    keys = keys_of(coords)
    lev = 5 if dense else 21
    L = O.Level(lev, keys, periodic_mask=7)
    ref = {int(k): i for i, k in enumerate(keys)}
    assert np.array_equal(L.lookup(keys), np.arange(len(keys), dtype=np.int32))
    q = keys_of(rng.integers(0, npd, size=(3000, 3), dtype=np.uint32))
    got = L.lookup(q)
    assert all(got[t] == ref.get(int(q[t]), -1) for t in range(len(q)))
    # linear-probing invariant: no empty slot between a key's home and its slot
    sk, sv = L.hash_dump()
    cap = len(sk)
    assert L.n <= 0.7 * cap
    empty = sk == np.uint64(0xFFFFFFFFFFFFFFFF)
    for s in np.nonzero(~empty)[0][:500]:
        home = O.hash_fn(int(sk[s])) & (cap - 1)
        t = home
        while t != s:
            assert not empty[t]
            t = (t + 1) % cap
        assert sv[s] == ref[int(sk[s])]


def test_build_errors():
    k = keys_of([[0, 0, 0], [1, 0, 0], [0, 0, 0]])
    with pytest.raises(O.OracleError) as e:
        O.Level(3, k)
    assert e.value.code == O.OR_ERR_DUPLICATE_KEY
    with pytest.raises(O.OracleError) as e:
        O.Level(2, keys_of([[2, 0, 0]]))  # level 2 has 2 octs per axis
    assert e.value.code == O.OR_ERR_KEY_OUT_OF_RANGE
    with pytest.raises(O.OracleError) as e:
        O.Level(3, np.array([1 << 63], dtype=np.uint64))
    assert e.value.code == O.OR_ERR_KEY_OUT_OF_RANGE


# --------------------------------------------------------- neighbour cache

@pytest.mark.parametrize("pmask", [7, 0, 5])
def test_neighbor_cache_bruteforce(pmask):
    rng = np.random.default_rng(4 + pmask)
    npd = 8
    coords = np.unique(rng.integers(0, npd, size=(300, 3), dtype=np.uint32), axis=0)
    rng.shuffle(coords)
    L = O.Level(4, keys_of(coords), periodic_mask=pmask)
    nb = L.neighbors()
    c = coords.astype(np.int64)
    for i in range(len(c)):
        assert nb[i, 0] == i
        for d in range(6):
            a, s = d // 2, (1 if d & 1 else -1)
            want = c[i].copy()
            want[a] += s
            if (pmask >> a) & 1:
                want[a] %= npd
            elif not 0 <= want[a] < npd:
                assert nb[i, 1 + d] == -1
                continue
            hit = np.nonzero(np.all(c == want, axis=1))[0]
            assert nb[i, 1 + d] == (hit[0] if len(hit) else -1)


def _two_level(base, seed=2):
    cfg = inputs.two_level_amr(base_level=base, seed=seed)
    B = O.Level(base, keys_of(cfg["coords"][0]))
    F = O.Level(base + 1, keys_of(cfg["coords"][1]), parent=B)
    return cfg, B, F


def test_father_cells_bruteforce():
    cfg, B, F = _two_level(4)
    fc = F.father_cells()
    nb = F.neighbors()
    pc = cfg["coords"][0].astype(np.int64)
    fcoords = cfg["coords"][1].astype(np.int64)
    npd = 1 << 4
    pos = {tuple(x): i for i, x in enumerate(pc)}
    for i in range(len(fcoords)):
        for d in range(6):
            if nb[i, 1 + d] >= 0:
                assert tuple(fc[i, d]) == (-1, -1)
                continue
            w = fcoords[i].copy()
            w[d // 2] = (w[d // 2] + (1 if d & 1 else -1)) % npd
            assert fc[i, d, 0] == pos[tuple(w >> 1)]
            assert fc[i, d, 1] == (w[0] & 1) + 2 * (w[1] & 1) + 4 * (w[2] & 1)


def test_mg_hierarchy_rule_bruteforce():
    cfg, B, F = _two_level(5)
    for m in range(F.mg_depth - 1):
        keys = F.mg_keys(m)
        act = F.mg_active(m)
        full = act.all(axis=1)
        parents = []
        seen = set()
        for k in keys[full]:
            p = int(k) >> 3
            if p not in seen:
                seen.add(p)
                parents.append(p)
        assert np.array_equal(F.mg_keys(m + 1), np.array(parents, dtype=np.uint64))
        cact = F.mg_active(m + 1)
        want = np.zeros_like(cact)
        ppos = {p: i for i, p in enumerate(parents)}
        for k in keys[full]:
            want[ppos[int(k) >> 3], int(k) & 7] = 1
        assert np.array_equal(cact, want)
        assert F.mg_lev(m + 1) == F.mg_lev(m) - 1
    # the top level is fully active; a full periodic level stays full down to one oct
    assert F.mg_active(0).all()
    assert [B.mg_n_octs(m) for m in range(B.mg_depth)] == [8 ** (4 - m) for m in range(5)]


# ------------------------------------------- operators vs dense formulation

def _periodic(level, seed=5):
    coords = inputs.uniform_oct_coords(level)
    L = O.Level(level, keys_of(coords))
    n = 1 << level
    rng = np.random.default_rng(seed)
    return L, coords, n, rng


def test_sweep_residual_vs_dense():
    L, coords, n, rng = _periodic(4)
    h = 1.0 / n
    phi = rng.standard_normal((n, n, n))
    f = rng.standard_normal((n, n, n))
    L.set_phi(inputs.dense_to_octs(phi, coords))
    L.set_f(inputs.dense_to_octs(f, coords))
    L.rb_sweeps(0, 1, use_ghost=False)
    want = D.rb_sweep(phi, f, h)
    assert np.array_equal(L.get_phi(), inputs.dense_to_octs(want, coords))
    n2 = L.residual(0, use_ghost=False)
    r = L.mg_get(0, "r")
    rd = D.residual(want, f, h)
    np.testing.assert_allclose(r, inputs.dense_to_octs(rd, coords), rtol=0, atol=1e-12 * np.abs(rd).max())
    assert abs(n2 - np.sum(rd * rd)) <= 1e-12 * np.sum(rd * rd)


def test_gauss_seidel_zeroes_the_residual_it_just_updated():
    """Red-black Gauss-Seidel solves each updated cell's equation exactly
    given its neighbours (App. D.2 Eq. (gs_update)), and the neighbours of a
    black cell are all red: after a sweep (red, then black) the residual
    vanishes on every black cell, up to rounding, while the red cells keep an
    O(|f|) residual.  Periodic 32^3 level and the refined level of a
    two-level pair (coarse-fine ghosts)."""
    L, coords, n, rng = _periodic(5)
    L.set_phi(rng.standard_normal((L.n, 8)))
    L.set_f(rng.standard_normal((L.n, 8)))
    levels = [(L, False)]
    cfg = inputs.two_level_amr(base_level=4, seed=3)
    B = O.Level(4, keys_of(cfg["coords"][0]))
    F = O.Level(5, keys_of(cfg["coords"][1]), parent=B)
    B.set_phi(rng.standard_normal((B.n, 8)))
    F.set_phi(rng.standard_normal((F.n, 8)))
    F.set_f(rng.standard_normal((F.n, 8)))
    levels.append((F, True))
    black = [c for c in range(8) if bin(c).count("1") % 2 == 1]
    red = [c for c in range(8) if bin(c).count("1") % 2 == 0]
    for G, ghost in levels:
        G.rb_sweeps(0, 1, use_ghost=ghost)
        G.residual(0, use_ghost=ghost)
        r = G.mg_get(0, "r")
        scale = np.abs(r[:, red]).max()
        assert scale > 0.1
        assert np.abs(r[:, black]).max() <= 1e-10 * scale


def test_restrict_prolong_vs_dense():
    L, coords, n, rng = _periodic(4)
    r = rng.standard_normal((n, n, n))
    L.mg_set(0, "r", inputs.dense_to_octs(r, coords))
    L.restrict(0)
    ccoords = O.morton_decode(L.mg_keys(1))
    got = inputs.octs_to_dense(L.mg_get(1, "f"), ccoords, n // 2)
    np.testing.assert_allclose(got, D.restrict(r), rtol=0, atol=1e-14)
    assert np.all(L.mg_get(1, "phi") == 0)
    e = rng.standard_normal((n // 2,) * 3)
    phi0 = rng.standard_normal((n, n, n))
    L.mg_set(1, "phi", inputs.dense_to_octs(e, ccoords))
    L.mg_set(0, "phi", inputs.dense_to_octs(phi0, coords))
    L.prolong(0)
    got = inputs.octs_to_dense(L.mg_get(0, "phi"), coords, n)
    np.testing.assert_allclose(got, phi0 + D.prolong(e), rtol=0, atol=1e-13)


def test_prolong_reproduces_linear_fields():
    # trilinear cell-centred interpolation is exact for linear fields away
    # from the periodic seam
    L, coords, n, rng = _periodic(4)
    ccoords = O.morton_decode(L.mg_keys(1)).astype(np.float64)
    hc = 2.0 / n

    def lin(x, y, z):
        return 0.3 + 1.7 * x - 0.9 * y + 2.3 * z

    off = inputs.child_offsets()
    Xc = (2 * ccoords[:, None, :] + off[None] + 0.5) * hc
    L.mg_set(1, "phi", lin(Xc[..., 0], Xc[..., 1], Xc[..., 2]))
    L.mg_set(0, "phi", np.zeros((L.n, 8)))
    L.prolong(0)
    fc = O.morton_decode(L.mg_keys(0)).astype(np.float64)
    h = 1.0 / n
    Xf = (2 * fc[:, None, :] + off[None] + 0.5) * h
    got = L.mg_get(0, "phi")
    inner = np.all((Xf > 1.5 * hc) & (Xf < 1 - 1.5 * hc), axis=2)
    want = lin(Xf[..., 0], Xf[..., 1], Xf[..., 2])
    np.testing.assert_allclose(got[inner], want[inner], rtol=0, atol=1e-13)


def test_wht_coarse_solve_vs_dense_matrix():
    L = O.Level(1, keys_of([[0, 0, 0]]))
    rng = np.random.default_rng(6)
    f = rng.standard_normal(8)
    f -= f.mean()
    L.set_f(f.reshape(1, 8))
    L.coarse_solve()
    phi = L.get_phi().ravel()
    # dense 2^3 periodic operator; child c = x + 2y + 4z -> dense index
    A = D.dense_matrix(2, 0.5)
    want = np.linalg.lstsq(A, _to_dense8(f), rcond=None)[0]
    want -= want.mean()
    np.testing.assert_allclose(_to_dense8(phi), want, rtol=0, atol=1e-13)


def _to_dense8(v):
    out = np.zeros(8)
    for c in range(8):
        out[np.ravel_multi_index(((c & 1), (c >> 1) & 1, (c >> 2) & 1), (2, 2, 2))] = v[c]
    return out


# --------------------------------------------------------- full solutions

def test_mg_matches_fft_solve():
    L, coords, n, rng = _periodic(4, seed=7)
    h = 1.0 / n
    f = rng.standard_normal((n, n, n))
    f -= f.mean()
    L.set_f(inputs.dense_to_octs(f, coords))
    rc, st = L.solve(tol=1e-13, max_cycles=60)
    got = inputs.octs_to_dense(L.get_phi(), coords, n)
    want = D.fft_solve(f, h)
    assert np.max(np.abs(got - want)) <= 1e-11 * np.max(np.abs(want))
    assert abs(got.mean()) < 1e-15 * np.abs(want).max() * n ** 3


def test_mg_matches_dense_solve_4cube():
    L, coords, n, rng = _periodic(2, seed=8)
    h = 1.0 / n
    f = rng.standard_normal((n, n, n))
    f -= f.mean()
    L.set_f(inputs.dense_to_octs(f, coords))
    L.solve(tol=1e-14, max_cycles=60)
    got = inputs.octs_to_dense(L.get_phi(), coords, n).ravel()
    want = np.linalg.lstsq(D.dense_matrix(n, h), f.ravel(), rcond=None)[0]
    want -= want.mean()
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.abs(want).max())


def _cell_centres(coords, level):
    off = inputs.child_offsets()
    h = 1.0 / (1 << level)
    X = (2 * coords[:, None, :].astype(np.float64) + off[None] + 0.5) * h
    return X[..., 0], X[..., 1], X[..., 2]


@pytest.mark.parametrize("level", [4, 5])
def test_paper_sine_mode_discrete_exact(level):
    """Sec. 8 Poisson microbenchmark source; the discrete solution is f / lambda_h."""
    coords = inputs.uniform_oct_coords(level)
    L = O.Level(level, keys_of(coords))
    x, y, z = _cell_centres(coords, level)
    s = np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y) * np.sin(2 * np.pi * z)
    f = -12 * np.pi ** 2 * s
    L.set_f(f)
    L.solve(tol=1e-12)
    h = 1.0 / (1 << level)
    lam = -(4 / h ** 2) * 3 * np.sin(np.pi * h) ** 2
    np.testing.assert_allclose(L.get_phi(), f / lam, rtol=0, atol=1e-10)


def test_paper_sine_mode_second_order():
    err = []
    for level in (4, 5, 6):
        coords = inputs.uniform_oct_coords(level)
        L = O.Level(level, keys_of(coords))
        x, y, z = _cell_centres(coords, level)
        s = np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y) * np.sin(2 * np.pi * z)
        L.set_f(-12 * np.pi ** 2 * s)
        L.solve(tol=1e-11)
        err.append(np.max(np.abs(L.get_phi() - s)))
    assert 3.8 < err[0] / err[1] < 4.2 and 3.9 < err[1] / err[2] < 4.1


def test_periodic_invariants_config1_small():
    cfg = inputs.periodic_grf_level(4, seed=1)
    coords = cfg["coords"][0]
    L = O.Level(4, keys_of(coords))
    rho = cfg["rho"][0]
    L.set_density(rho, rho.mean())
    f = L.get_f()
    assert abs(f.sum()) < 1e-12 * np.abs(f).sum()
    rc, st = L.solve(tol=1e-10)
    phi = L.get_phi()
    assert abs(phi.mean()) < 1e-14 * np.abs(phi).max()
    n = 1 << 4
    r = D.residual(inputs.octs_to_dense(phi, coords, n), inputs.octs_to_dense(f, coords, n), 1.0 / n)
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(f)
    assert st["rel_final"] <= 1e-10
    assert st["cycles"] <= 14


def test_vcycle_convergence_factor():
    cfg = inputs.periodic_grf_level(5, seed=1)
    L = O.Level(5, keys_of(cfg["coords"][0]))
    L.set_density(cfg["rho"][0], 1.0)
    rc, st = L.solve(tol=1e-10)
    h = np.array(st["rel_history"])
    assert np.all(h[1:] / h[:-1] < 0.15)


# ------------------------------------------------ refined (Dirichlet) levels

def _patch(level, lo, hi):
    """Octs of a cube patch [lo, hi) in box units at the given level."""
    npd = 1 << (level - 1)
    a, b = int(round(lo * npd)), int(round(hi * npd))
    r = np.arange(a, b)
    z, y, x = np.meshgrid(r, r, r, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], 1).astype(np.uint32)


def _patch_problem(level, phi_fn, f_fn):
    pc = inputs.uniform_oct_coords(level - 1)
    P = O.Level(level - 1, keys_of(pc))
    x, y, z = _cell_centres(pc, level - 1)
    P.set_phi(phi_fn(x, y, z))
    fc = _patch(level, 0.25, 0.75)
    F = O.Level(level, keys_of(fc), parent=P)
    x, y, z = _cell_centres(fc, level)
    F.set_f(f_fn(x, y, z))
    return P, F, (x, y, z)


def test_ghosts_exact_for_linear_parent():
    lin = lambda x, y, z: 0.25 - 1.5 * x + 0.75 * y + 2.0 * z  # noqa: E731
    P, F, _ = _patch_problem(5, lin, lambda x, y, z: 0 * x)
    g = F.ghosts()
    nb = F.neighbors()
    fc = O.morton_decode(F.mg_keys(0)).astype(np.float64)
    h = 1.0 / 32
    n_checked = 0
    for i in range(F.n):
        for d in range(6):
            if nb[i, 1 + d] >= 0:
                assert np.all(np.isnan(g[i, d]))
                continue
            a, side = d // 2, d & 1
            q = 0
            for c in range(8):
                if ((c >> a) & 1) != side:
                    continue
                X = 2 * fc[i] + np.array([c & 1, (c >> 1) & 1, (c >> 2) & 1])
                X[a] += 1 if side else -1
                xc = (X + 0.5) * h
                assert abs(g[i, d, q] - lin(*xc)) < 1e-13
                q += 1
                n_checked += 1
    # a 8^3-oct cube patch has 6 faces of 8 x 8 octs, 4 ghost cells each
    assert n_checked == 6 * 8 * 8 * 4


def _plummer(a=0.1, M=1.0):
    def phi(x, y, z):
        r2 = (x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2
        return -M / np.sqrt(r2 + a * a)

    def f(x, y, z):  # 4 pi G rho with G = 1
        r2 = (x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2
        rho = 3 * M / (4 * np.pi * a ** 3) * (1 + r2 / a ** 2) ** -2.5
        return 4 * np.pi * rho

    return phi, f


def test_plummer_patch_second_order():
    phi, f = _plummer()
    err = []
    for level in (5, 6):
        P, F, X = _patch_problem(level, phi, f)
        rc, st = F.solve(tol=1e-11)
        err.append(np.max(np.abs(F.get_phi() - phi(*X))))
    assert 3.3 < err[0] / err[1] < 4.7, err


def test_uniform_sphere_patch():
    R, rho0 = 0.15, 1.0
    M = 4 / 3 * np.pi * R ** 3 * rho0

    def phi(x, y, z):
        r = np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2)
        return np.where(r < R, -2 * np.pi * rho0 * (R ** 2 - r ** 2 / 3), -M / np.maximum(r, 1e-300))

    def f(x, y, z):
        r = np.sqrt((x - 0.5) ** 2 + (y - 0.5) ** 2 + (z - 0.5) ** 2)
        return np.where(r < R, 4 * np.pi * rho0, 0.0)

    P, F, X = _patch_problem(6, phi, f)
    F.solve(tol=1e-11)
    err = np.max(np.abs(F.get_phi() - phi(*X)))
    assert err < 0.02 * np.max(np.abs(phi(*X)))


def test_two_level_smooth_mode_second_order():
    """A refined region over a smooth periodic field reproduces the continuum
    solution to O(h^2), interface included (base solved first, then the fine
    level with ghosts interpolated from it)."""
    err = []
    for base in (4, 5):
        cfg = inputs.two_level_amr(base_level=base, seed=2)
        cb, cf = cfg["coords"]
        B = O.Level(base, keys_of(cb))
        x, y, z = _cell_centres(cb, base)
        s = np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y) * np.sin(2 * np.pi * z)
        B.set_f(-12 * np.pi ** 2 * s)
        B.solve(tol=1e-12)
        F = O.Level(base + 1, keys_of(cf), parent=B)
        x, y, z = _cell_centres(cf, base + 1)
        s = np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y) * np.sin(2 * np.pi * z)
        F.set_f(-12 * np.pi ** 2 * s)
        F.solve(tol=1e-12)
        err.append(np.max(np.abs(F.get_phi() - s)))
    assert 3.3 < err[0] / err[1] < 4.7, err


def test_missing_parent_error():
    pc = _patch(4, 0.25, 0.75)
    P = O.Level(4, keys_of(pc), periodic_mask=7)
    fc = _patch(5, 0.25, 0.75)  # the patch reaches the edge of its parent patch
    with pytest.raises(O.OracleError) as e:
        O.Level(5, keys_of(fc), parent=P)
    assert e.value.code == O.OR_ERR_MISSING_PARENT


def test_not_converged_status():
    cfg = inputs.periodic_grf_level(4, seed=1)
    L = O.Level(4, keys_of(cfg["coords"][0]))
    L.set_density(cfg["rho"][0], 1.0)
    rc, st = L.solve(tol=1e-10, max_cycles=2, raise_on_error=False)
    assert rc == O.OR_ERR_NOT_CONVERGED and st["cycles"] == 2


def test_mixed_precision_converges_to_fp64():
    cfg, B, F = _two_level(5)
    B.set_density(cfg["rho"][0], 1.0)
    B.solve(tol=1e-13)
    F.set_density(cfg["rho"][1], 1.0)
    F.solve(tol=1e-13)
    ref = F.get_phi()
    F.set_phi(np.zeros_like(ref))
    rc, st = F.solve_mixed(tol=1e-10)
    got = F.get_phi()
    assert st["rel_final"] <= 1e-10
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref))
