"""Square-free factorisation of a polynomial in Z[x] -- test infrastructure only.

The paper's solver computes, for each resultant polynomial R, a square-free
factorisation of it (Section 5, the PROJECT phase).  The plain definition: R = c * prod_i R_i^i
with c in Z, every R_i in Z[x] primitive with positive leading coefficient,
square-free, and the R_i pairwise coprime; constant factors are omitted.

The steps are Yun's algorithm (D. Y. Y. Yun, "On square-free decomposition
algorithms", SYMSAC 1976), taken over Z with primitive polynomials so that
every division is exact (Gauss's lemma):
    A = gcd(F, F'),  B = F / A,  C = F' / A,  D = C - B';
    repeat: R_i = gcd(B, D), B = B / R_i, C = D / R_i, D = C - B'
    until deg B = 0.
Polynomial gcds are taken by the primitive remainder sequence (pseudo-
remainders made primitive after every step).  Polynomials are lists of ints,
index = power of x, no trailing zeros.
"""
from math import gcd

from .exact import zx_divexact, zx_mul, zx_sub, zx_trim


def derivative(a):
    return zx_trim([i * a[i] for i in range(1, len(a))])


def content(a):
    c = 0
    for v in a:
        c = gcd(c, v)
    return c


def primitive(a):
    """The primitive part with a positive leading coefficient ([] for 0)."""
    a = zx_trim(a)
    if not a:
        return []
    c = content(a)
    if a[-1] < 0:
        c = -c
    return [v // c for v in a]


def pseudo_rem(a, b):
    """lc(b)^(deg a - deg b + 1) a mod b, computed by row operations."""
    a = list(a)
    db, lb = len(b) - 1, b[-1]
    while len(a) - 1 >= db and a:
        la, s = a[-1], len(a) - 1 - db
        a = [lb * v for v in a]
        for i, v in enumerate(b):
            a[s + i] -= la * v
        a = zx_trim(a)
    return a


def zx_gcd(a, b):
    """Primitive gcd with positive leading coefficient (gcd(0, 0) = [])."""
    a, b = primitive(a), primitive(b)
    if len(a) < len(b):
        a, b = b, a
    while b:
        a, b = b, primitive(pseudo_rem(a, b))
    return a


def squarefree(R):
    """(c, [(i, R_i), ...]) with R = c * prod R_i^i as described above, the
    factors in increasing multiplicity.  R must be non-zero."""
    R = zx_trim(R)
    if not R:
        raise ValueError("square-free factorisation of 0")
    F = primitive(R)
    c = R[-1] // F[-1]
    if len(F) == 1:
        return c, []
    A = zx_gcd(F, derivative(F))
    B = zx_divexact(F, A)
    C = zx_divexact(derivative(F), A)
    D = zx_sub(C, derivative(B))
    out, i = [], 1
    while len(B) > 1:
        Ri = zx_gcd(B, D)
        B = zx_divexact(B, Ri)
        C = zx_divexact(D, Ri)
        D = zx_sub(C, derivative(B))
        if len(Ri) > 1:
            out.append((i, Ri))
        i += 1
    return c, out


def expand(c, factors):
    """c * prod R_i^i."""
    out = [c]
    for i, Ri in factors:
        for _ in range(i):
            out = zx_mul(out, Ri)
    return out
