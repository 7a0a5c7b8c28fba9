"""Property tests of the oracle's level build on random key sets (dense,
sparse, touching the box boundary, around the hash-capacity edges): every key
found at its index, absent keys missing, fill <= 0.7 in a power-of-two table,
and every neighbour and father cell equal to plain coordinate arithmetic."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import oracle as O  # noqa: E402


@st.composite
def key_sets(draw):
    level = draw(st.integers(2, 7))
    npd = 1 << (level - 1)
    n_max = min(npd ** 3, 400)
    # sizes around the capacity edges (0.7 * 2^k) as well as random ones
    edge = [k for k in (11, 12, 22, 23, 44, 45, 89, 90, 179, 180, 358, 359) if k <= n_max]
    n = draw(st.one_of(st.sampled_from(edge or [1]), st.integers(1, n_max)))
    seed = draw(st.integers(0, 2 ** 31 - 1))
    rng = np.random.default_rng(seed)
    flat = rng.choice(npd ** 3, size=n, replace=False)
    coords = np.stack([flat % npd, (flat // npd) % npd, flat // (npd * npd)], 1).astype(np.uint32)
    pmask = draw(st.sampled_from([0, 1, 3, 7]))
    return level, coords, pmask


@settings(max_examples=60, deadline=None)
@given(key_sets())
def test_random_key_sets(case):
    level, coords, pmask = case
    npd = 1 << (level - 1)
    keys = O.morton_encode(coords)
    R = O.Level(level, keys, periodic_mask=pmask)
    cap = R.hash_capacity
    assert cap & (cap - 1) == 0 and 10 * len(keys) <= 7 * cap and (cap == 1 or 10 * len(keys) > 7 * (cap // 2))
    assert np.array_equal(R.lookup(keys), np.arange(len(keys)))
    pos = {tuple(int(v) for v in c): i for i, c in enumerate(coords)}
    absent = np.array([[x, y, z] for x in range(npd) for y in range(npd) for z in range(npd)
                       if (x, y, z) not in pos][:50], dtype=np.uint32).reshape(-1, 3)
    if len(absent):
        assert np.all(R.lookup(O.morton_encode(absent)) == -1)
    nb = R.neighbors()
    for i, c in enumerate(coords):
        for d in range(6):
            y = [int(v) for v in c]
            a = d // 2
            y[a] += 1 if d & 1 else -1
            if (pmask >> a) & 1:
                y[a] %= npd
            want = pos.get(tuple(y), -1) if 0 <= y[a] < npd else -1
            assert nb[i, 1 + d] == want
