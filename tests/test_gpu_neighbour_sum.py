"""The FP64 neighbour sum every stencil kernel forms (Sec. 5.1.1's 7-point
update sums the six face neighbours), checked on its own through
cmg_debug_neighbour_sum, bit for bit.

The library sums operands as integers at the scale 2^(E - 1082) (E the
largest biased exponent among them) and rounds that sum once to nearest
(ties to even): the first five neighbours, then one FP64 addition of the
sixth, in colour passes and colour-1 residuals (which = 0); all six in
colour-0 residuals (which = 1).  Two checks pin it to something other than
its own description:

* Rows whose integer-summed operands are all multiples of that scale (in
  particular, within seven binades of one another) are summed exactly, so
  the integer step must equal Python's math.fsum, the correctly rounded sum.
  Ties, exact cancellations and signed mixtures are built in on purpose.
* Any row: the result must equal an exact-arithmetic model of the same rule
  (Python integers and correctly rounded int -> float conversion), and lie
  within half an ulp plus the five truncations of the exact sum.

Zeros are compared without their sign (the integer sum has no -0), NaN by
being NaN."""
import math
import struct

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__ as ge
    ge.build()
    from paper_2604_06035_gb300 import cmg
    c = cmg.cmg_ctx_create(0)
    yield c
    cmg.cmg_ctx_destroy(c)


def _bits(x):
    return struct.unpack("<Q", struct.pack("<d", float(x)))[0]


def _biased_exp(x):
    return (_bits(x) >> 52) & 0x7FF


def _fixed_model(v):
    """The integer-scaled sum of FP64 values, in exact arithmetic."""
    es = [_biased_exp(x) for x in v]
    E = max(es)
    if E >= 0x7FC or E < 64:
        s = float(v[0])
        for x in v[1:]:
            s = s + float(x)
        return s
    S = 0
    for x, e in zip(v, es):
        if e == 0:  # zero or subnormal: far below the scale
            continue
        m = (_bits(x) & ((1 << 52) - 1)) | (1 << 52)  # |x| = m 2^(e - 1075)
        k = E - e - 7  # |x| / 2^(E - 1082) = m 2^-k
        t = m >> k if k >= 0 else m << -k  # truncated toward zero
        S += -t if x < 0 else t
    sh = E - 1082
    return float(S * (1 << sh)) if sh >= 0 else S / (1 << -sh)


def _model(row, which):
    if which == 0:
        return _fixed_model(row[:5]) + float(row[5])
    return _fixed_model(row[:6])


def _same(a, b):
    a, b = float(a), float(b)
    if math.isnan(a) or math.isnan(b):
        return math.isnan(a) and math.isnan(b)
    if a == 0.0 and b == 0.0:
        return True
    return _bits(a) == _bits(b)


def _gpu(ctx, rows, which):
    import torch
    from paper_2604_06035_gb300 import cmg
    rows = np.ascontiguousarray(rows, dtype=np.float64)
    out = cmg.cmg_debug_neighbour_sum(ctx, torch.from_numpy(rows).cuda(), which)
    host = cmg.cmg_debug_neighbour_sum(ctx, rows, which)
    got = out.cpu().numpy()
    assert np.array_equal(got.view(np.uint64), np.asarray(host).view(np.uint64))
    return got


def _exact_rows(rng, n, k):
    """Rows whose first k (5 or 6) operands are multiples of the scale; with
    k = 5 the sixth is a random value of similar size."""
    rows = []
    for _ in range(n):
        kind = rng.integers(5)
        base = math.ldexp(1.0, int(rng.integers(-300, 300)))
        if kind == 0:  # same binade range: random significands, mixed signs
            r = [float(x) * base for x in rng.uniform(-2, 2, k)]
            r = [x if abs(x) >= base / 64 else base / 3 for x in r]
        elif kind == 1:  # exact cancellation leaving a small remainder
            a, b = (float(x) * base for x in rng.uniform(1, 2, 2))
            r = [a, -a, b, -b, base * 2.0 ** -int(rng.integers(0, 7))] + [-base] * (k - 5)
        elif kind == 2:  # a tie: 1 + half an ulp (+ further half ulps)
            one = base * (1.0 + math.ldexp(float(rng.integers(2)), -52))
            h = math.ldexp(base, -53)
            r = [one, h, 0.0, -0.0, 0.0] if rng.integers(2) else [one, h, h, -h, 0.0]
            r += [0.0] * (k - 5)
        elif kind == 3:  # integers far apart in size (exact at the scale)
            r = [float(int(x)) * base for x in rng.integers(-2**20, 2**20, k)]
            r[0] = base * 2.0 ** 21
        else:  # the sum carries into a higher binade and ties there (2.5 ulps)
            r = [base * (2.0 - math.ldexp(1.0, -52))] * 4 + [3 * math.ldexp(base, -49)] + [0.0] * (k - 5)
        rng.shuffle(r)
        rows.append(r + [float(rng.normal()) * base] * (6 - k))
    return np.array(rows, dtype=np.float64)


def _general_rows(rng, n):
    e = rng.integers(-90, 90, size=(n, 6))
    rows = rng.uniform(1, 2, size=(n, 6)) * np.exp2(e) * rng.choice([-1.0, 1.0], size=(n, 6))
    # some rows at level-solve magnitudes, some with a far smaller sixth value
    rows[: n // 4] = rng.normal(size=(n // 4, 6))
    rows[n // 4: n // 2, 5] *= 1e-30
    special = [
        [0.0] * 6,
        [-0.0] * 6,
        [5e-324, -5e-324, 1e-310, 2.2e-308, 0.0, 1.0],  # five subnormals: FP64 additions
        [1.0, 5e-324, -1e-310, 2.2e-308, -0.0, 0.0],  # subnormals beside a normal value vanish
        [1e-300, 5e-324, -3e-310, 0.0, 0.0, 0.0],  # all below 2^-960: FP64 additions
        [math.inf, 1.0, 2.0, 3.0, 4.0, 5.0],
        [-math.inf, math.inf, 0.0, 0.0, 0.0, 0.0],
        [math.nan, 1.0, 0.0, 0.0, 0.0, 0.0],
        [1.7e308, 1.7e308, -1.0, 0.0, 0.0, 0.0],  # >= 2^1021: FP64 additions, overflow to inf
        [math.ldexp(1.0, 1020) * 1.9] * 5 + [0.0],  # just under 2^1021: integers, near the top
        [1.0, 2.0 ** -60, 2.0 ** -61, 3 * 2.0 ** -62, -(2.0 ** -59), 0.0],  # truncated bits
    ]
    return np.concatenate([rows, np.array(special)])


@pytest.mark.parametrize("which", [0, 1])
def test_exact_rows_match_the_correctly_rounded_sum(ctx, which):
    k = 5 if which == 0 else 6
    rows = _exact_rows(np.random.default_rng(7 + which), 4000, k)
    got = _gpu(ctx, rows, which)
    for r, g in zip(rows, got):
        want = math.fsum(r[:5]) + r[5] if which == 0 else math.fsum(r)
        assert _same(g, want), (list(r), g, want)


@pytest.mark.parametrize("which", [0, 1])
def test_every_row_matches_the_exact_model(ctx, which):
    rows = _general_rows(np.random.default_rng(8), 20000)
    got = _gpu(ctx, rows, which)
    for r, g in zip(rows, got):
        assert _same(g, _model(r, which)), (list(r), g, _model(r, which))


@pytest.mark.parametrize("which", [0, 1])
def test_error_bound_against_the_exact_sum(ctx, which):
    """|integer-scaled sum - exact| <= half an ulp of the result + one
    truncation per operand, each below 2^(E - 1082), on rows with operands
    spread over 180 binades."""
    from fractions import Fraction
    k = 5 if which == 0 else 6
    rows = _general_rows(np.random.default_rng(9), 3000)[:3000]
    if which == 0:
        rows[:, 5] = 0.0  # the sixth enters as +0.0: out is the five-operand sum
    got = _gpu(ctx, rows, which)
    for r, g in zip(rows, got):
        E = max(_biased_exp(x) for x in r[:k])
        if E < 64:
            continue
        exact = sum(Fraction(float(x)) for x in r[:k])
        ulp = Fraction(math.ulp(float(g))) if g != 0 else Fraction(0)
        bound = ulp / 2 + k * Fraction(2) ** (E - 1082)
        assert abs(Fraction(float(g)) - exact) <= bound, list(r)


@pytest.mark.parametrize("which", [0, 1])
def test_order_of_the_integer_summed_operands_does_not_matter(ctx, which):
    k = 5 if which == 0 else 6
    rng = np.random.default_rng(10)
    rows = _general_rows(rng, 2000)[:2000]
    perm = rows.copy()
    for r in perm:
        r[:k] = r[rng.permutation(k)]
    a, b = _gpu(ctx, rows, which), _gpu(ctx, perm, which)
    assert all(_same(x, y) for x, y in zip(a, b))


def test_argument_checks(ctx):
    from paper_2604_06035_gb300 import cmg
    with pytest.raises(ValueError):
        cmg.cmg_debug_neighbour_sum(ctx, np.zeros(7))
    with pytest.raises(cmg.CmgError):
        cmg.cmg_debug_neighbour_sum(ctx, np.zeros((2, 6)), which=2)
    assert cmg.cmg_debug_neighbour_sum(ctx, np.zeros((0, 6))).shape == (0,)


@pytest.mark.parametrize("which", [0, 1])
def test_signed_zeros_bit_for_bit(ctx, which):
    """Rows of zeros of every sign pattern: the integer sums return at once
    with the sign sequential FP64 additions give (-0 only when every summed
    operand is -0), compared bit for bit."""
    import itertools
    rows = np.array([list(sg) for sg in itertools.product([0.0, -0.0], repeat=6)], dtype=np.float64)
    got = _gpu(ctx, rows, which)
    for r, g in zip(rows, got):
        s = float(r[0])
        for x in r[1:]:
            s = s + float(x)  # sequential FP64 additions: the same value and sign here
        assert _bits(g) == _bits(s), (list(r), g, s)
