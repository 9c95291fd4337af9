"""Exact resultant R^{(y)} = res(f, g, y) in Z[x] -- test infrastructure only.

Definitions followed (paper, Section 2 and Section 3.1):

* Eq. (2.1): f = sum f_ij x^i y^j.  Here a bivariate polynomial is a
  rectangular list ``f[i][j]`` of Python ints, i the x-exponent and j the
  y-exponent (zero entries allowed).  Written as a polynomial in y,
  f = sum_{j=0}^{m_y} f_j^{(y)}(x) y^j with f_j^{(y)} in Z[x] and m_y the
  y-degree.
* Section 3.1: R^{(y)} is the determinant of the (m_y+n_y) x (m_y+n_y)
  Sylvester matrix whose first n_y rows hold f_{m_y}^{(y)}, ..., f_0^{(y)}
  (descending powers of y), each row shifted one column to the right of the
  previous one, followed by m_y rows built the same way from g.
* Section 3.1: deg R^{(y)} <= m * n (total degrees).

Conventions where the paper is silent (the paper assumes f, g non-zero and
coprime): f == 0 or g == 0 gives R = 0; m_y = n_y = 0 gives the empty
determinant 1.

A univariate polynomial in Z[x] is a list of ints, index = power of x, with
no trailing zeros ([] is the zero polynomial).
"""
from fractions import Fraction
from itertools import permutations

# ---------------------------------------------------------------- Z[x] ring


def zx_trim(a):
    a = list(a)
    while a and a[-1] == 0:
        a.pop()
    return a


def zx_add(a, b):
    n = max(len(a), len(b))
    return zx_trim([(a[i] if i < len(a) else 0) + (b[i] if i < len(b) else 0)
                    for i in range(n)])


def zx_neg(a):
    return [-c for c in a]


def zx_sub(a, b):
    return zx_add(a, zx_neg(b))


def zx_mul(a, b):
    if not a or not b:
        return []
    out = [0] * (len(a) + len(b) - 1)
    for i, ai in enumerate(a):
        if ai:
            for j, bj in enumerate(b):
                out[i + j] += ai * bj
    return zx_trim(out)


def zx_divexact(a, b):
    """Quotient of a by b in Z[x]; raises if b does not divide a exactly."""
    a = zx_trim(a)
    b = zx_trim(b)
    if not b:
        raise ZeroDivisionError("division by the zero polynomial")
    q = [0] * max(len(a) - len(b) + 1, 0)
    r = list(a)
    lb = b[-1]
    for k in range(len(q) - 1, -1, -1):
        c = r[k + len(b) - 1]
        if c % lb:
            raise ArithmeticError("inexact division in Z[x]")
        c //= lb
        q[k] = c
        if c:
            for i, bi in enumerate(b):
                r[k + i] -= c * bi
    if any(r):
        raise ArithmeticError("inexact division in Z[x]")
    return zx_trim(q)


def zx_eval(a, x0):
    v = 0
    for c in reversed(a):
        v = v * x0 + c
    return v


ZX = dict(zero=[], one=[1], is_zero=lambda a: not a, mul=zx_mul, sub=zx_sub,
          divexact=zx_divexact, neg=zx_neg)


def _int_divexact(a, b):
    q, r = divmod(a, b)
    if r:
        raise ArithmeticError("inexact integer division")
    return q


ZZ = dict(zero=0, one=1, is_zero=lambda a: a == 0, mul=lambda a, b: a * b,
          sub=lambda a, b: a - b, divexact=_int_divexact, neg=lambda a: -a)

# ------------------------------------------------------- input and matrix


def is_zero_bipoly(f):
    return not any(c for row in f for c in row)


def y_coefficients(f):
    """[f_0^{(y)}, ..., f_{m_y}^{(y)}] as Z[x] polynomials (Eq. (2.1))."""
    if is_zero_bipoly(f):
        return []
    ny = max(len(row) for row in f)
    cols = [zx_trim([row[j] if j < len(row) else 0 for row in f]) for j in range(ny)]
    while cols and not cols[-1]:
        cols.pop()
    return cols


def sylvester(fy, gy):
    """Sylvester matrix S^{(y)}(f, g) of Section 3.1 with Z[x] entries."""
    my, ny = len(fy) - 1, len(gy) - 1
    r = my + ny
    S = [[[] for _ in range(r)] for _ in range(r)]
    for row in range(ny):  # f-rows: f_{m_y}, ..., f_0 starting at column `row`
        for k in range(my + 1):
            S[row][row + k] = list(fy[my - k])
    for row in range(my):  # g-rows: g_{n_y}, ..., g_0 starting at column `row`
        for k in range(ny + 1):
            S[ny + row][row + k] = list(gy[ny - k])
    return S


def map_matrix(M, fn):
    return [[fn(e) for e in row] for row in M]

# ------------------------------------------------------------ determinants


def _perm_sign(p):
    p = list(p)
    s = 1
    for i in range(len(p)):
        while p[i] != i:
            j = p[i]
            p[i], p[j] = p[j], p[i]
            s = -s
    return s


def det_leibniz(M, ring=ZZ):
    """sum over permutations sigma of sign(sigma) prod_i M[i][sigma(i)]."""
    n = len(M)
    total = ring["zero"]
    for p in permutations(range(n)):
        term = ring["one"]
        for i in range(n):
            term = ring["mul"](term, M[i][p[i]])
            if ring["is_zero"](term):
                break
        if ring["is_zero"](term):
            continue
        total = ring["sub"](total, term) if _perm_sign(p) < 0 else \
            ring["sub"](total, ring["neg"](term))
    return total


def det_bareiss(M, ring=ZZ):
    """Fraction-free (Bareiss) elimination over an integral domain with exact
    division; row swaps for zero pivots."""
    n = len(M)
    if n == 0:
        return ring["one"]
    A = [list(row) for row in M]
    sign = 1
    prev = ring["one"]
    for k in range(n - 1):
        if ring["is_zero"](A[k][k]):
            sw = next((i for i in range(k + 1, n) if not ring["is_zero"](A[i][k])), None)
            if sw is None:
                return ring["zero"]
            A[k], A[sw] = A[sw], A[k]
            sign = -sign
        akk = A[k][k]
        for i in range(k + 1, n):
            aik = A[i][k]
            for j in range(k + 1, n):
                num = ring["sub"](ring["mul"](A[i][j], akk), ring["mul"](aik, A[k][j]))
                A[i][j] = ring["divexact"](num, prev)
        prev = akk
    d = A[n - 1][n - 1]
    return d if sign > 0 else ring["neg"](d)

# ---------------------------------------------------------------- bounds


def degree_bound(f, g):
    """deg R^{(y)} <= m * n with m, n the total degrees (Section 3.1)."""
    def tdeg(h):
        return max((i + j for i, row in enumerate(h) for j, c in enumerate(row) if c),
                   default=-1)
    return max(tdeg(f), 0) * max(tdeg(g), 0)


def hadamard_square(fy, gy):
    """H^2 >= |det M(x)|^2 on |x| = 1 for M = S^{(y)} or any square minor of
    it: product over rows of sum_j ||f_j||_1^2 (each factor >= 1 here)."""
    my, ny = len(fy) - 1, len(gy) - 1
    rf = sum(sum(abs(c) for c in fj) ** 2 for fj in fy)
    rg = sum(sum(abs(c) for c in gj) ** 2 for gj in gy)
    return rf ** ny * rg ** my

# ------------------------------------------------------------ resultants


def _degenerate(f, g):
    fy, gy = y_coefficients(f), y_coefficients(g)
    if not fy or not gy:
        return None, None, []
    return fy, gy, None


def resultant_y_leibniz(f, g):
    """det S^{(y)}(f, g) by permutation expansion over Z[x] (tiny r only)."""
    fy, gy, z = _degenerate(f, g)
    if z is not None:
        return z
    return det_leibniz(sylvester(fy, gy), ZX)


def resultant_y_bareiss_zx(f, g):
    """det S^{(y)}(f, g) by Bareiss with exact division in Z[x]."""
    fy, gy, z = _degenerate(f, g)
    if z is not None:
        return z
    return det_bareiss(sylvester(fy, gy), ZX)


def resultant_y(f, g):
    """det S^{(y)}(f, g) via the Kronecker map x -> 2^k (a ring homomorphism
    Z[x] -> Z, injective on polynomials whose coefficients lie in
    (-2^(k-1), 2^(k-1))): integer Bareiss on S(2^k), then unpack in signed
    base 2^k.  k is chosen from the Hadamard bound, which bounds every minor
    met by the elimination, so pivots vanish exactly when the polynomial
    pivots do and the final image unpacks uniquely."""
    fy, gy, z = _degenerate(f, g)
    if z is not None:
        return z
    h2 = hadamard_square(fy, gy)
    k = (h2.bit_length() + 1) // 2 + 2
    X = 1 << k
    S = map_matrix(sylvester(fy, gy), lambda e: zx_eval(e, X))
    v = det_bareiss(S, ZZ)
    out = []
    half, mask = 1 << (k - 1), X - 1
    while v:
        d = v & mask
        if d >= half:
            d -= X
        out.append(d)
        v = (v - d) >> k
    return zx_trim(out)


def transpose(f):
    """The same polynomial with the two variables exchanged: rows indexed by
    the y-exponent, entries by the x-exponent."""
    nx = len(f)
    ny = max((len(r) for r in f), default=0)
    return [[f[i][j] if j < len(f[i]) else 0 for i in range(nx)] for j in range(ny)]


def resultant_x(f, g):
    """R^{(x)} = res(f, g, x) in Z[y] (Section 3.1: defined like R^{(y)}, with
    f and g read as polynomials in x whose coefficients lie in Z[y]).  After
    exchanging the variables the Sylvester determinant is taken exactly as
    for R^{(y)}; the result's coefficient k belongs to y^k."""
    return resultant_y(transpose(f), transpose(g))


def resultant_y_at(f, g, x0):
    """R^{(y)}(x0) = det S^{(y)}(f(x0, y), g(x0, y)) in Z (evaluation commutes
    with the determinant because the formal y-degrees are kept)."""
    fy, gy, z = _degenerate(f, g)
    if z is not None:
        return 0
    S = map_matrix(sylvester(fy, gy), lambda e: zx_eval(e, x0))
    return det_bareiss(S, ZZ)


def interpolate_consecutive(values):
    """The polynomial P in Q[x] of degree < len(values) with P(i) = values[i]
    (i = 0, 1, ...), returned with integer coefficients (raises if P is not
    in Z[x]).  Newton form on the points 0..D: P = sum_k (Delta^k v_0 / k!)
    x (x-1) ... (x-k+1), expanded to monomials."""
    D = len(values) - 1
    diffs = list(values)
    lead = [diffs[0]]
    for _ in range(D):
        diffs = [diffs[i + 1] - diffs[i] for i in range(len(diffs) - 1)]
        lead.append(diffs[0])
    acc = [Fraction(0)] * (D + 1)
    falling = [1]  # x (x-1) ... (x-k+1)
    fact = 1
    for k in range(D + 1):
        if k:
            fact *= k
            falling = zx_sub([0] + falling, [(k - 1) * c for c in falling]) or []
            falling = falling + [0] * (k + 1 - len(falling))
        ck = Fraction(lead[k], fact)
        if ck:
            for i, c in enumerate(falling):
                acc[i] += ck * c
    out = []
    for c in acc:
        if c.denominator != 1:
            raise ArithmeticError("interpolant is not in Z[x]")
        out.append(c.numerator)
    return zx_trim(out)


def resultant_y_interp(f, g, pool=None):
    """R^{(y)} from its exact values at x = 0..D, D = degree_bound(f, g)
    (Section 3.1), by exact interpolation.  ``pool`` is an optional
    ``multiprocessing`` pool used to evaluate the points in parallel."""
    fy, gy, z = _degenerate(f, g)
    if z is not None:
        return z
    D = degree_bound(f, g)
    xs = list(range(D + 1))
    if pool is None:
        vals = [resultant_y_at(f, g, x) for x in xs]
    else:
        vals = pool.starmap(resultant_y_at, [(f, g, x) for x in xs])
    return interpolate_consecutive(vals)
