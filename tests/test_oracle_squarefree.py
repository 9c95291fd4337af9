"""Pins of the oracle's square-free factorisation (oracle/squarefree.py):
planted products c * P1 * P2^2 * P3^3 of square-free, pairwise coprime
factors come back exactly; the factors of any input multiply back to it and
are square-free and pairwise coprime; sympy's sqf_list agrees on random
inputs (a library special case); a Yun step done wrong is caught."""
import random

import pytest

from oracle import exact, squarefree as sq
from oracle.exact import zx_mul

sympy = pytest.importorskip("sympy")


def rand_poly(rng, deg, bound=9):
    p = [rng.randint(-bound, bound) for _ in range(deg)] + [rng.choice([-3, -2, -1, 1, 2, 3])]
    return p


def sympy_sqf(R):
    x = sympy.Symbol("x")
    P = sympy.Poly(list(reversed(R)), x, domain="ZZ")
    c, facs = P.sqf_list()
    out = []
    for fac, mult in facs:
        co = [int(v) for v in reversed(fac.all_coeffs())]
        if co[-1] < 0:  # sympy's factors may have a negative leading coefficient
            co = [-v for v in co]
            if mult % 2:
                c = -c
        out.append((mult, co))
    return int(c), sorted(out)


def is_squarefree_and_coprime(factors):
    for _, P in factors:
        if sq.zx_gcd(P, sq.derivative(P)) != [1]:
            return False
    for a in range(len(factors)):
        for b in range(a + 1, len(factors)):
            if sq.zx_gcd(factors[a][1], factors[b][1]) != [1]:
                return False
    return True


def test_planted_products():
    rng = random.Random(61)
    done = 0
    while done < 12:
        P = [sq.primitive(rand_poly(rng, rng.randint(1, 4))) for _ in range(3)]
        if not is_squarefree_and_coprime([(1, p) for p in P]):
            continue
        c = rng.choice([1, -1, 6, -35, 2 ** 40 + 1])
        R = [c]
        for i, p in enumerate(P, start=1):
            for _ in range(i):
                R = zx_mul(R, p)
        assert sq.squarefree(R) == (c, [(1, P[0]), (2, P[1]), (3, P[2])])
        done += 1


def test_invariants_and_sympy_agree():
    rng = random.Random(62)
    for _ in range(25):
        R = [rng.choice([-2, 3])]
        for _ in range(rng.randint(1, 4)):
            f = rand_poly(rng, rng.randint(1, 3))
            for _ in range(rng.randint(1, 3)):
                R = zx_mul(R, f)
        c, facs = sq.squarefree(R)
        assert sq.expand(c, facs) == R
        assert is_squarefree_and_coprime(facs)
        assert all(P[-1] > 0 and sq.content(P) == 1 for _, P in facs)
        assert [m for m, _ in facs] == sorted(m for m, _ in facs)
        assert (c, sorted(facs)) == sympy_sqf(R)


def test_square_free_input_and_constants():
    assert sq.squarefree([5]) == (5, [])
    assert sq.squarefree([-4, 0, 2]) == (2, [(1, [-2, 0, 1])])
    assert sq.squarefree([0, 0, 3]) == (3, [(2, [0, 1])])  # 3 x^2
    with pytest.raises(ValueError):
        sq.squarefree([])


def test_resultant_with_a_repeated_factor():
    """Res_y(p q^2, g) = Res_y(p, g) Res_y(q, g)^2 (multiplicativity): the
    square-free factorisation of a resultant with a planted square."""
    rng = random.Random(63)
    p = [[rng.randint(-3, 3) for _ in range(3)] for _ in range(2)]
    q = [[rng.randint(-3, 3) for _ in range(2)] for _ in range(2)]
    p[1][2] = q[1][1] = 1
    from paper_1010_1386_gb300.inputs import _dy, _from_dict, _mul_dict, _to_dict
    pq = _mul_dict(_to_dict(p), _to_dict(q))
    f = _from_dict(_mul_dict(pq, _to_dict(q)))
    g = _from_dict(_dy(pq))
    R = exact.resultant_y(f, g)
    c, facs = sq.squarefree(R)
    assert sq.expand(c, facs) == R
    Rq = exact.resultant_y(q, g)
    if Rq and len(Rq) > 1:  # the square of Res_y(q, g) shows up with multiplicity >= 2
        assert any(m >= 2 for m, _ in facs)


def test_planted_yun_mistake_is_caught():
    """Yun with the gcd taken against C instead of D = C - B' fails the
    planted products."""
    def wrong(R):
        F = sq.primitive(R)
        A = sq.zx_gcd(F, sq.derivative(F))
        B = exact.zx_divexact(F, A)
        C = exact.zx_divexact(sq.derivative(F), A)
        out, i = [], 1
        while len(B) > 1 and i < 6:
            Ri = sq.zx_gcd(B, C)
            B = exact.zx_divexact(B, Ri)
            C = exact.zx_divexact(C, Ri) if len(Ri) > 1 else C
            if len(Ri) > 1:
                out.append((i, Ri))
            i += 1
        return R[-1] // F[-1], out
    P = [[1, 1], [-2, 0, 1], [3, 1, 1]]  # x + 1, x^2 - 2, x^2 + x + 3
    R = zx_mul(zx_mul(P[0], zx_mul(P[1], P[1])), zx_mul(P[2], zx_mul(P[2], P[2])))
    assert sq.squarefree(R) == (1, [(1, P[0]), (2, P[1]), (3, P[2])])
    assert wrong(R) != sq.squarefree(R)
