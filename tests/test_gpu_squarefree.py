"""Square-free factorisation of Res_y(f, g) through rs_squarefree_y against
the oracle (exact resultant, then Yun over Z): pairs whose resultant has
planted repeated factors (f = p q^2 with g = d(pq)/dy gives Res_y(p, g)
Res_y(q, g)^2), random pairs (square-free resultants), a degree-0 and a zero
resultant, too small a max_mult; and the non-generic workload at full size
checked by expanding the factors back to the GPU resultant."""
import random

import pytest

from oracle import exact, squarefree as sq
from paper_1010_1386_gb300 import inputs, rs
from paper_1010_1386_gb300.inputs import _dy, _from_dict, _mul_dict, _to_dict
from tests.helpers import rand_bipoly

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = rs.Context(device=0)
    yield c
    c.close()


def _trim_mod(a):
    while a and a[-1] == 0:
        a.pop()
    return a


def _deriv_mod(a, q):
    return _trim_mod([i * a[i] % q for i in range(1, len(a))])


def _gcd_mod(a, b, q):
    """Monic gcd of polynomials mod a prime q (ascending lists)."""
    a, b = _trim_mod(list(a)), _trim_mod(list(b))
    while b:
        inv = pow(b[-1], q - 2, q)
        while len(a) >= len(b):
            t, s = a[-1] * inv % q, len(a) - len(b)
            for i, v in enumerate(b):
                a[s + i] = (a[s + i] - t * v) % q
            _trim_mod(a)
        a, b = b, a
    inv = pow(a[-1], q - 2, q)
    return [v * inv % q for v in a]


def planted(rng, dp, dq, bits):
    p = rand_bipoly(rng, dp, dp, bits=bits)
    q = rand_bipoly(rng, dq, dq, bits=bits)
    pq = _mul_dict(_to_dict(p), _to_dict(q))
    f = _from_dict(_mul_dict(pq, _to_dict(q)))
    g = _from_dict(_dy(pq))
    return f, g


def test_planted_repeated_factors_exact(ctx):
    rng = random.Random(71)
    for dp, dq, bits in [(1, 1, 4), (2, 1, 6), (2, 1, 20), (3, 1, 8), (2, 2, 5)]:
        f, g = planted(rng, dp, dq, bits)
        want = sq.squarefree(exact.resultant_y(f, g))
        got = ctx.squarefree(f, g)
        assert got == want, (dp, dq, bits)
        assert any(m >= 2 for m, _ in got[1])


def test_random_pairs_exact(ctx):
    rng = random.Random(72)
    for _ in range(12):
        f = rand_bipoly(rng, rng.randint(1, 4), rng.randint(1, 4), bits=rng.choice([4, 30, 70]))
        g = rand_bipoly(rng, rng.randint(1, 4), rng.randint(1, 4), bits=rng.choice([4, 30, 70]))
        R = exact.resultant_y(f, g)
        if not R:
            continue
        assert ctx.squarefree(f, g) == sq.squarefree(R)


def test_constant_zero_and_multiplicity_limit(ctx):
    assert ctx.squarefree([[3]], [[0, 1]]) == (3, [])          # Res_y(3, y) = 3
    with pytest.raises(rs.RsError) as ei:
        ctx.squarefree([[0, 1]], [[0, 2]])                     # Res_y(y, 2y) = 0
    assert ei.value.code == -1
    f = [[0, 1]]                                               # f = y
    g = [[0, 0, 0, 1], [0], [0], [-1]]                         # g = y^3 - x^3: Res_y(y, g) = -x^3
    assert ctx.squarefree(f, g) == (-1, [(3, [0, 1])])
    with pytest.raises(rs.RsError) as ei:
        ctx.squarefree(f, g, max_mult=2)
    assert ei.value.code == -2


def test_nongeneric_workload_full_size(ctx):
    """The first pair of the coprime topology workload (f = p q^2, g =
    d(pq)/dy, total degrees 48 and 35): the factors multiply back to the GPU
    resultant.  By multiplicativity R = Res_y(p, g) Res_y(q, g)^2, which is
    disc_y(p) disc_y(q)^2 Res_y(p, q)^3 up to a constant, so factors of
    multiplicities 1, 2 and 3 appear."""
    (f, g), = inputs.workload_nongeneric(3, n=1, coprime=True)
    R = ctx.resultant_y(f, g)
    c, facs = ctx.squarefree(f, g)
    assert sq.expand(c, facs) == R
    # square-free and pairwise coprime: a common factor over Z would survive
    # reduction mod a prime that divides no leading coefficient
    q = (1 << 61) - 1
    assert all(P[-1] % q for _, P in facs)
    red = [[v % q for v in P] for _, P in facs]
    for i, A in enumerate(red):
        assert len(_gcd_mod(A, _deriv_mod(A, q), q)) == 1
        for B in red[i + 1:]:
            assert len(_gcd_mod(A, B, q)) == 1
    assert all(P[-1] > 0 for _, P in facs) and [m for m, _ in facs] == sorted(m for m, _ in facs)
    assert [m for m, _ in facs] == [1, 2, 3]
    info = ctx.squarefree_info()  # every primitive part passed the device check
    assert info["factors"] == 3 and info["factors_device"] == 3


def test_batch_mixed_pairs(ctx):
    """One pass over planted, random, constant and zero resultants: every
    pair matches the oracle, the zero one fails alone with RS_ERR_ARG."""
    rng = random.Random(73)
    pairs = [planted(rng, dp, dq, bits) for dp, dq, bits in [(2, 1, 9), (1, 2, 3), (3, 2, 12)]]
    pairs += [(rand_bipoly(rng, 3, 3, bits=40), rand_bipoly(rng, 2, 4, bits=5)) for _ in range(3)]
    pairs += [([[3]], [[0, 1]]), ([[0, 1]], [[0, 2]]), ([[0, 1]], [[0, 0, 0, 1], [0], [0], [-1]])]
    got = ctx.squarefree_batch(pairs)
    info = ctx.squarefree_info()
    assert info["factors"] > 0 and info["factors_device"] == info["factors"]
    for i, ((f, g), r) in enumerate(zip(pairs, got)):
        R = exact.resultant_y(f, g)
        if not R:
            assert isinstance(r, rs.RsError) and r.code == -1, i
        else:
            assert r == sq.squarefree(R), i


def test_both_projections_in_one_pass(ctx):
    """rs_squarefree_projections: Res_y and Res_x of each pair factored in one
    pass, each equal to the oracle's factorisation of the oracle's
    resultant in that variable."""
    rng = random.Random(74)
    pairs = [planted(rng, 2, 1, 7), planted(rng, 1, 1, 5)]
    pairs += [(rand_bipoly(rng, 3, 2, bits=20), rand_bipoly(rng, 2, 3, bits=9))]
    got = ctx.squarefree_projections(pairs)
    for (f, g), (sy, sx) in zip(pairs, got):
        assert sy == sq.squarefree(exact.resultant_y(f, g))
        assert sx == sq.squarefree(exact.resultant_x(f, g))


def test_hand_derived_content_sign_and_factors(ctx):
    """Res_y(y - x, g) = g(x, x); with g = -6 (y - 1)^2 (x + 2) this is
    R = -6 (x - 1)^2 (x + 2): content -6 (the sign of lc R), x + 2 with
    multiplicity 1 and x - 1 with multiplicity 2."""
    f = [[0, 1], [-1, 0]]  # y - x  (f[i][j]: coefficient of x^i y^j)
    # -6 (y^2 - 2y + 1)(x + 2) = -12 + 24 y - 12 y^2 - 6 x + 12 x y - 6 x y^2
    g = [[-12, 24, -12], [-6, 12, -6]]
    want = (-6, [(1, [2, 1]), (2, [-1, 1])])
    assert sq.squarefree(exact.resultant_y(f, g)) == want
    assert ctx.squarefree(f, g) == want
