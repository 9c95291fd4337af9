"""Pins for the CPU oracle, against facts that do not come from the oracle:
hand-derived worked examples (tests/golden), brute-force permutation
expansion, the product formula for the resultant, antisymmetry and
multiplicativity, sympy's Sylvester determinant on tiny inputs, the degree and Hadamard
bounds, and planted common roots.  A final group plants mistakes in the
oracle and checks that these pins catch them."""
import glob
import os
import random

import numpy as np
import pytest

from oracle import exact, modp
from oracle.exact import zx_add, zx_mul, zx_trim
from tests.helpers import ALL_GOLDEN, GOLDEN, GOLDEN_X, from_factors, golden_var, load_golden, subst_y  # noqa: F401

HERE = os.path.dirname(os.path.abspath(__file__))


def rand_bipoly(rng, dx, dy, bound=20, density=1.0):
    f = [[(rng.randint(-bound, bound) if rng.random() < density else 0) for _ in range(dy + 1)]
         for _ in range(dx + 1)]
    if f[dx][dy] == 0:
        f[dx][dy] = 1
    return f





@pytest.mark.parametrize("path", GOLDEN, ids=[os.path.basename(p) for p in GOLDEN])
def test_golden(path):
    f, g, R = load_golden(path)
    assert exact.resultant_y_leibniz(f, g) == R
    assert exact.resultant_y_bareiss_zx(f, g) == R
    assert exact.resultant_y(f, g) == R
    assert exact.resultant_y_interp(f, g) == R


@pytest.mark.parametrize("path", GOLDEN_X, ids=[os.path.basename(p) for p in GOLDEN_X])
def test_golden_resultant_x(path):
    f, g, R = load_golden(path)
    assert exact.resultant_x(f, g) == R


def test_resultant_x_product_formula_and_projections():
    """Res_x(f, g) = lc_x(f)^{n_x} prod_i g(a_i(y), y) for f = c * prod_i (x - a_i(y))
    with a_i in Z[y]; and both projections vanish at the coordinates of a
    planted common root (Theorem 3.1)."""
    rng = random.Random(41)
    for trial in range(6):
        c = rng.choice([1, -2, 3])
        roots = [[rng.randint(-3, 3) for _ in range(rng.randint(1, 3))] for _ in range(rng.randint(1, 3))]
        # f(x, y) = c * prod (x - a_i(y)) as rows f[i][j] (x^i y^j)
        fx = [[c]]  # coefficients in x, each a Z[y] polynomial
        for a in roots:
            nxt = [[] for _ in range(len(fx) + 1)]
            for i, ci in enumerate(fx):
                nxt[i + 1] = zx_add(nxt[i + 1], ci)
                nxt[i] = zx_add(nxt[i], zx_mul([-1], zx_mul(a, ci)))
            fx = nxt
        f = exact.transpose(exact.transpose([list(r) for r in fx]))  # rows by x-exponent
        g = rand_bipoly(rng, rng.randint(1, 3), rng.randint(0, 3))
        R = exact.resultant_x(f, g)
        # prod_i g(a_i(y), y): evaluate g at x = a_i(y) in Z[y]
        want = [c ** (len(g) - 1)] if len(g) > 1 else [1]
        for a in roots:
            val = []
            for i, row in enumerate(g):
                term = list(row)
                for _ in range(i):
                    term = zx_mul(term, a)
                val = zx_add(val, term)
            want = zx_mul(want, val)
        assert R == zx_trim(want), trial
    # planted common root (x0, y0) = (2, -1)
    f = [[1, 0, 1], [0, 1, 0], [-1, 0, 0]]        # 1 + y^2 + x y - x^2 -> f(2,-1) = 1 + 1 - 2 - 4 != 0
    f[0][0] -= (1 + 1 - 2 - 4)                    # shift so that f(2, -1) = 0
    g = [[3, 1], [1, 0]]                          # 3 + y + x -> g(2, -1) = 4
    g[0][0] -= 4
    Ry, Rx = exact.resultant_y(f, g), exact.resultant_x(f, g)
    assert exact.zx_eval(Ry, 2) == 0 and exact.zx_eval(Rx, -1) == 0
    assert Ry and Rx


def test_planted_transpose_mistake_is_caught():
    """An x-projection that forgot to exchange the variables is caught by the
    worked examples."""
    wrong = [exact.resultant_y(*load_golden(p)[:2]) == load_golden(p)[2] for p in GOLDEN_X]
    assert not all(wrong)


def test_leibniz_bareiss_kronecker_interp_agree():
    rng = random.Random(11)
    for _ in range(40):
        dx1, dy1, dx2, dy2 = (rng.randint(0, 3) for _ in range(4))
        if dy1 + dy2 > 6:
            continue
        f = rand_bipoly(rng, dx1, dy1, density=0.7)
        g = rand_bipoly(rng, dx2, dy2, density=0.7)
        ref = exact.resultant_y_leibniz(f, g)
        assert exact.resultant_y_bareiss_zx(f, g) == ref
        assert exact.resultant_y(f, g) == ref
        assert exact.resultant_y_interp(f, g) == ref


@pytest.mark.parametrize("seed", range(6))
def test_product_formula(seed):
    """Res_y(f, g) = a^{n_y} prod_i g(x, alpha_i(x)) for f = a prod (y - alpha_i)."""
    rng = random.Random(100 + seed)
    a = [rng.randint(-5, 5) for _ in range(rng.randint(1, 3))]
    a[-1] = a[-1] or 2
    alphas = [[rng.randint(-4, 4) for _ in range(rng.randint(1, 3))] for _ in range(rng.randint(1, 4))]
    f = from_factors(a, alphas)
    g = rand_bipoly(rng, rng.randint(0, 3), rng.randint(1, 4), bound=9)
    ny = len(exact.y_coefficients(g)) - 1
    expect = [1]
    for _ in range(ny):
        expect = zx_mul(expect, zx_trim(a))
    for al in alphas:
        expect = zx_mul(expect, subst_y(g, al))
    assert exact.resultant_y(f, g) == expect
    assert exact.resultant_y_interp(f, g) == expect
    if len(alphas) + ny <= 6:
        assert exact.resultant_y_leibniz(f, g) == expect


@pytest.mark.parametrize("seed", range(5))
def test_antisymmetry_and_multiplicativity(seed):
    rng = random.Random(200 + seed)
    f = rand_bipoly(rng, rng.randint(0, 3), rng.randint(1, 4))
    g = rand_bipoly(rng, rng.randint(0, 3), rng.randint(1, 3))
    h = rand_bipoly(rng, rng.randint(0, 2), rng.randint(1, 3))
    my, ny = len(exact.y_coefficients(f)) - 1, len(exact.y_coefficients(g)) - 1
    rfg, rgf = exact.resultant_y(f, g), exact.resultant_y(g, f)
    assert rfg == ([-c for c in rgf] if (my * ny) % 2 else rgf)
    gh = [[0] * (len(g[0]) + len(h[0]) - 1) for _ in range(len(g) + len(h) - 1)]
    for i1, r1 in enumerate(g):
        for j1, c1 in enumerate(r1):
            for i2, r2 in enumerate(h):
                for j2, c2 in enumerate(r2):
                    gh[i1 + i2][j1 + j2] += c1 * c2
    assert exact.resultant_y(f, gh) == zx_mul(rfg, exact.resultant_y(f, h))


def test_sympy_special_case():
    """sympy's own Sylvester matrix (subresultants_qq_zz.sylvester) and its
    determinant.  (sympy.resultant itself is not used: for deg_y f = 1 and odd
    deg_y g it returns the negative of its own Sylvester determinant.)"""
    sympy = pytest.importorskip("sympy")
    from sympy.polys.subresultants_qq_zz import sylvester
    x, y = sympy.symbols("x y")
    rng = random.Random(7)
    for _ in range(12):
        f = rand_bipoly(rng, rng.randint(0, 3), rng.randint(1, 5))
        g = rand_bipoly(rng, rng.randint(0, 3), rng.randint(1, 5))
        F = sum(c * x ** i * y ** j for i, r in enumerate(f) for j, c in enumerate(r))
        G = sum(c * x ** i * y ** j for i, r in enumerate(g) for j, c in enumerate(r))
        det = sympy.expand(sympy.Matrix(sylvester(F, G, y)).det())
        ref = sympy.Poly(det, x).all_coeffs()[::-1] if det != 0 else []
        assert exact.resultant_y(f, g) == zx_trim([int(c) for c in ref])


def test_degree_and_hadamard_bounds():
    rng = random.Random(5)
    for _ in range(10):
        f = rand_bipoly(rng, rng.randint(1, 4), rng.randint(1, 4), bound=1000)
        g = rand_bipoly(rng, rng.randint(1, 4), rng.randint(1, 4), bound=1000)
        R = exact.resultant_y(f, g)
        assert len(R) - 1 <= exact.degree_bound(f, g)
        h2 = exact.hadamard_square(exact.y_coefficients(f), exact.y_coefficients(g))
        assert all(c * c <= h2 for c in R)


def test_planted_common_root():
    rng = random.Random(9)
    for _ in range(6):
        x0, y0 = rng.randint(-3, 3), rng.randint(-3, 3)
        f = rand_bipoly(rng, 2, 2)
        g = rand_bipoly(rng, 2, 3)
        f[0][0] -= sum(c * x0 ** i * y0 ** j for i, r in enumerate(f) for j, c in enumerate(r))
        g[0][0] -= sum(c * x0 ** i * y0 ** j for i, r in enumerate(g) for j, c in enumerate(r))
        R = exact.resultant_y(f, g)
        assert exact.zx_eval(R, x0) == 0
        assert exact.resultant_y_at(f, g, x0) == 0


def test_modp_image_matches_exact():
    rng = random.Random(3)
    primes = [2147483647, 2147483629, 1073741827, 998244353]
    for _ in range(8):
        f = rand_bipoly(rng, rng.randint(0, 4), rng.randint(1, 5), bound=10 ** 6)
        g = rand_bipoly(rng, rng.randint(0, 4), rng.randint(1, 5), bound=10 ** 6)
        R = exact.resultant_y(f, g)
        for p in primes:
            x0 = rng.randint(0, p - 1)
            assert modp.resultant_image(f, g, p, x0) == exact.zx_eval(R, x0) % p


def test_modp_det_bruteforce():
    rng = random.Random(4)
    p = 1000003
    for n in range(1, 6):
        M = [[rng.randint(-50, 50) for _ in range(n)] for _ in range(n)]
        assert modp.det_mod_p(M, p) == exact.det_leibniz(M) % p


def test_conventions():
    f0 = [[0, 0], [0, 0]]
    g = [[1, 2], [3, 4]]
    assert exact.resultant_y(f0, g) == [] and exact.resultant_y(g, f0) == []
    # m_y = 0: R = f^{n_y} (Sylvester matrix = f_0 * identity of size n_y)
    f = [[2], [3]]  # 2 + 3x
    g = rand_bipoly(random.Random(1), 2, 3)
    assert exact.resultant_y(f, g) == zx_mul(zx_mul([2, 3], [2, 3]), [2, 3])
    assert exact.resultant_y(g, f) == zx_mul(zx_mul([2, 3], [2, 3]), [2, 3])
    assert exact.resultant_y([[5]], [[7], [1]]) == [1]


# ---- planted mistakes: each must be caught by the pins above -------------

def _bad_sylvester_g_first(fy, gy):
    my, ny = len(fy) - 1, len(gy) - 1
    r = my + ny
    S = [[[] for _ in range(r)] for _ in range(r)]
    for row in range(my):
        for k in range(ny + 1):
            S[row][row + k] = list(gy[ny - k])
    for row in range(ny):
        for k in range(my + 1):
            S[my + row][row + k] = list(fy[my - k])
    return S


def _bad_sylvester_ascending(fy, gy):
    my, ny = len(fy) - 1, len(gy) - 1
    r = my + ny
    S = [[[] for _ in range(r)] for _ in range(r)]
    for row in range(ny):
        for k in range(my + 1):
            S[row][row + k] = list(fy[k])
    for row in range(my):
        for k in range(ny + 1):
            S[ny + row][row + k] = list(gy[k])
    return S


@pytest.mark.parametrize("bad", [_bad_sylvester_g_first, _bad_sylvester_ascending])
def test_planted_mistakes_are_caught(monkeypatch, bad):
    monkeypatch.setattr(exact, "sylvester", bad)
    caught = False
    for path in GOLDEN:
        f, g, R = load_golden(path)
        caught |= exact.resultant_y(f, g) != R
    rng = random.Random(100)
    for seed in range(6):
        rng = random.Random(100 + seed)
        a = [rng.randint(-5, 5) for _ in range(rng.randint(1, 3))]
        a[-1] = a[-1] or 2
        alphas = [[rng.randint(-4, 4) for _ in range(rng.randint(1, 3))]
                  for _ in range(rng.randint(1, 4))]
        f = from_factors(a, alphas)
        g = rand_bipoly(rng, rng.randint(0, 3), rng.randint(1, 4), bound=9)
        ny = len(exact.y_coefficients(g)) - 1
        expect = [1]
        for _ in range(ny):
            expect = zx_mul(expect, zx_trim(a))
        for al in alphas:
            expect = zx_mul(expect, subst_y(g, al))
        caught |= exact.resultant_y(f, g) != expect
    assert caught


def test_planted_dropped_term_is_caught(monkeypatch):
    orig = exact.zx_eval

    def dropped(a, x0):  # forgets the constant term
        return orig([0] + list(a[1:]), x0) if a else 0
    monkeypatch.setattr(exact, "zx_eval", dropped)
    f, g, R = load_golden(GOLDEN[0])
    bad = [exact.resultant_y(*load_golden(p)[:2]) != load_golden(p)[2] for p in GOLDEN]
    assert any(bad)


def test_generator_roundtrip():
    from paper_1010_1386_gb300 import inputs
    rng = np.random.Generator(np.random.PCG64(0))
    for bits, L in [(16, 1), (32, 1), (33, 2), (64, 2), (100, 4), (128, 4)]:
        a = inputs.signed_uniform_limbs(rng, (500,), bits, L)
        vals = [int.from_bytes(r.astype("<u4").tobytes(), "little", signed=True) for r in a]
        assert min(vals) >= -(1 << (bits - 1)) and max(vals) < (1 << (bits - 1))
        assert min(vals) < -(1 << (bits - 3)) and max(vals) > (1 << (bits - 3))
    rows = [[0, -5, 1 << 70], [-(1 << 90), 3, 0]]
    assert inputs.BiPoly.from_ints(rows).to_ints() == rows
