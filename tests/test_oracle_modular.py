"""Pins of the independent modular oracle O2 (``oracle/modres.c``).

O2 is pinned to things other than itself: the exact oracle O1 (Kronecker
map + integer Bareiss, and its stored digests at sizes O1 needs minutes
for), the worked examples of Section 3.1, the closed form
Res_y(a prod (y - alpha_i), g) = a^{n_y} prod g(x, alpha_i(x)), the
invariants Res(f, g) = (-1)^{m_y n_y} Res(g, f) and Res(f, g h) =
Res(f, g) Res(f, h), numpy Gaussian elimination of the Sylvester matrix mod
p for single images, Python's own integers for the Chinese remaindering, and
sympy's prime generator for the prime table.  Seven planted mistakes (O2
compiled with O2_PLANT = 1..7) must each fail the pins.
"""
import json
import os
import random
import sys

import numpy as np
import pytest

from oracle import exact, modp, modular
from paper_1010_1386_gb300 import inputs
from tests.helpers import ALL_GOLDEN, GOLDEN_DIR, from_factors, golden_var, load_golden, rand_bipoly, subst_y

TOP = (1 << 31) - (1 << 20)


def _pairs(seed, n, dmax=5, bits=(4, 20, 40, 90)):
    rng = random.Random(seed)
    out = []
    for _ in range(n):
        f = rand_bipoly(rng, rng.randint(0, dmax), rng.randint(0, dmax + 1), bits=rng.choice(bits))
        g = rand_bipoly(rng, rng.randint(0, dmax), rng.randint(0, dmax + 1), bits=rng.choice(bits))
        out.append((f, g))
    return out


def _unlucky_pair(rng):
    """lc_y f = x (x - 1) (x - 2) vanishes at the points 0, 1, 2 for every
    prime; m_y = 3, n_y = 5 (odd product, so a row-order mistake shows)."""
    f = rand_bipoly(rng, 3, 3, bits=30)
    f[0][3], f[1][3], f[2][3], f[3][3] = 0, 2, -3, 1
    g = rand_bipoly(rng, 2, 5, bits=30)
    return f, g


def _unlucky_prime_pair(rng, p):
    """lc_y f the constant p: every point is unlucky for the prime p."""
    f = rand_bipoly(rng, 2, 3, bits=30)
    f[0][3], f[1][3], f[2][3] = p, 0, 0
    g = rand_bipoly(rng, 3, 2, bits=30)
    return f, g


def _pin_set(rng):
    """Pairs every planted mistake must fail on: random small pairs with
    negative coefficients, the unlucky-point pair, m_y = 0 and n_y = 0."""
    pairs = _pairs(rng.randrange(1 << 30), 24)
    pairs.append(_unlucky_pair(rng))
    pairs.append((rand_bipoly(rng, 3, 0, bits=20), rand_bipoly(rng, 2, 3, bits=20)))
    pairs.append((rand_bipoly(rng, 2, 3, bits=20), rand_bipoly(rng, 3, 0, bits=20)))
    return pairs


# ------------------------------------------------------------ prime table

def test_prime_table():
    sympy = pytest.importorskip("sympy")
    table = [modular.prime(k) for k in range(8192)]
    assert modular.prime(8192) == 0 and modular.prime(-1) == 0
    assert all(a > b for a, b in zip(table, table[1:]))
    assert table[0] < TOP and table[-1] > (1 << 30)
    # no prime skipped: the table is every prime of [table[-1], TOP), descending
    want = sorted(sympy.primerange(table[299], TOP), reverse=True)
    assert table[:300] == want
    assert all(sympy.isprime(p) for p in table[::97])
    # and none of them is one of the GPU library's primes (all above TOP)
    assert table[0] == max(sympy.primerange(TOP - 200, TOP))


# ----------------------------------------------------------- against O1

def test_random_small_pairs_match_o1():
    pairs = _pairs(3, 150)
    got = modular.resultants(pairs, threads=4)
    for (f, g), R in zip(pairs, got):
        assert R == exact.resultant_y(f, g)


def test_worked_examples():
    for path in ALL_GOLDEN:
        f, g, R = load_golden(path)
        if golden_var(path) == "x":
            assert modular.resultant(exact.transpose(f), exact.transpose(g)) == R, path
        else:
            assert modular.resultant(f, g) == R, path


def test_conventions_and_degenerate_inputs():
    zero = [[0, 0], [0, 0]]
    h = rand_bipoly(random.Random(2), 2, 3)
    assert modular.resultant(zero, h) == [] and modular.resultant(h, zero) == []
    assert modular.resultant([[5]], [[7], [1]]) == [1]  # m_y = n_y = 0: the empty determinant
    f0 = [[2], [3]]  # m_y = 0: R = f^{n_y}
    assert modular.resultant(f0, h) == exact.resultant_y(f0, h)
    assert modular.resultant(h, f0) == exact.resultant_y(h, f0)
    padded = [row + [0, 0] for row in h] + [[0] * (len(h[0]) + 2)]
    assert modular.resultant(padded, f0) == exact.resultant_y(h, f0)
    # a common factor (y - x): R = 0
    rng = random.Random(3)
    a, b = rand_bipoly(rng, 2, 2), rand_bipoly(rng, 1, 3)

    def times_y_minus_x(p):
        out = [[0] * (len(p[0]) + 1) for _ in range(len(p) + 1)]
        for i, row in enumerate(p):
            for j, c in enumerate(row):
                out[i][j + 1] += c
                out[i + 1][j] -= c
        return out
    assert modular.resultant(times_y_minus_x(a), times_y_minus_x(b)) == []


def test_unlucky_points_and_prime_match_o1():
    rng = random.Random(4)
    f, g = _unlucky_pair(rng)
    assert modular.resultant(f, g) == exact.resultant_y(f, g)
    p0 = modular.prime(0)
    for x in (0, 1, 2):
        with pytest.raises(RuntimeError):
            modular.image(f, g, p0, x, how=2)  # the Euclidean branch refuses: lc vanishes
        assert modular.image(f, g, p0, x) == modp.resultant_image(f, g, p0, x)
    f, g = _unlucky_prime_pair(rng, p0)
    assert modular.resultant(f, g) == exact.resultant_y(f, g)


def test_small_configs_and_stored_o1_digests():
    [(f, g)] = inputs.workload_small(0)
    assert modular.resultant(f, g) == exact.resultant_y(f.to_ints(), g.to_ints())
    path = os.path.join(GOLDEN_DIR, "o1_pins.json")
    o1 = json.load(open(path))["workloads"]
    sys.path.insert(0, GOLDEN_DIR)
    from make_full_size import workloads
    checked = 0
    for name, done in o1.items():
        if name == "c0_small":
            continue
        pairs = workloads()[name][1]()
        idx = sorted(int(i) for i in done)
        got = modular.resultants([pairs[i] for i in idx], threads=8)
        for i, R in zip(idx, got):
            assert modular.digest(R) == done[str(i)]["sha256"], f"{name}[{i}]"
            checked += 1
    assert "0" in o1["c1_single"] and checked >= 3


# --------------------------------------------------- closed forms, invariants

@pytest.mark.parametrize("seed", range(3))
def test_product_formula(seed):
    """f = a(x) prod_{i<m} (y - alpha_i(x)): Res_y(f, g) = a^{n_y} prod g(x, alpha_i(x))
    in plain Z[x] arithmetic, at sizes O1 would need minutes for."""
    rng = random.Random(100 + seed)
    m, n = (12, 8) if seed else (16, 10)
    a = [rng.randint(-30, 30) for _ in range(3)]
    a[-1] = a[-1] or 5
    alphas = [[rng.randint(-30, 30), rng.randint(-30, 30) or 1] for _ in range(m)]
    f = from_factors(a, alphas)
    g = rand_bipoly(rng, 6, n, bits=24)
    want = [1]
    for _ in range(n):
        want = exact.zx_mul(want, exact.zx_trim(a))
    for al in alphas:
        want = exact.zx_mul(want, subst_y(g, al))
    assert modular.resultant(f, g) == want


def test_antisymmetry_and_multiplicativity():
    rng = random.Random(7)
    for _ in range(4):
        f = rand_bipoly(rng, rng.randint(2, 8), rng.randint(3, 12), bits=40)
        g = rand_bipoly(rng, rng.randint(2, 8), rng.randint(3, 12), bits=40)
        h = rand_bipoly(rng, rng.randint(1, 4), rng.randint(1, 5), bits=20)
        my, ny = len(f[0]) - 1, len(g[0]) - 1
        Rfg, Rgf = modular.resultants([(f, g), (g, f)])
        assert Rgf == [(-1) ** (my * ny) * c for c in Rfg]
        gh = [[0] * (len(g[0]) + len(h[0]) - 1) for _ in range(len(g) + len(h) - 1)]
        for i, row in enumerate(g):
            for j, c in enumerate(row):
                for k, row2 in enumerate(h):
                    for l2, d in enumerate(row2):
                        gh[i + k][j + l2] += c * d
        Rfgh, Rfh = modular.resultants([(f, gh), (f, h)])
        assert Rfgh == exact.zx_mul(Rfg, Rfh)


# --------------------------------------------------------- the three steps

def test_images_both_branches_match_gaussian_elimination():
    rng = random.Random(8)
    primes = [modular.prime(0), modular.prime(5), 1000000007, 998244353, 2147483647]
    for f, g in _pairs(9, 30, dmax=6):
        for p in primes:
            x = rng.randrange(p)
            want = modp.resultant_image(f, g, p, x)
            assert modular.image(f, g, p, x, how=1) == want
            assert modular.image(f, g, p, x, how=0) == want
            try:
                assert modular.image(f, g, p, x, how=2) == want
            except RuntimeError:
                pass  # a leading coefficient vanishes at x mod p: no Euclid image


def test_residues_are_o1_mod_p():
    for f, g in _pairs(10, 25):
        R = exact.resultant_y(f, g)
        for p in (modular.prime(3), 1000000007):
            got = modular.residues(f, g, p)
            want = [(R[i] if i < len(R) else 0) % p for i in range(len(got))]
            assert got == want
            assert len(got) >= len(R)  # the degree bound holds


def test_crt_matches_python_integers():
    rng = random.Random(12)
    for K in (1, 2, 5, 40, 300):
        ps = [modular.prime(k) for k in range(K)]
        P = 1
        for p in ps:
            P *= p
        vals = [rng.randrange(-(P // 2), P // 2 + 1) for _ in range(20)]
        vals += [0, 1, -1, P // 2, -(P // 2)]
        res = [[v % p for v in vals] for p in ps]
        res.append([0] * len(vals))  # unused row: the call takes K = len(res)
        got = modular.crt(res[:K], bits=31 * K)
        assert got == vals
        # residues at the edges of each prime's range
        edge = [[(p - 1) if c % 3 == 0 else ((p + 1) // 2 if c % 3 == 1 else (p - 1) // 2) for c in range(9)]
                for p in ps]
        want = []
        for c in range(9):
            x, M = 0, 1
            for k, p in enumerate(ps):
                x += M * (((edge[k][c] - x) * pow(M, -1, p)) % p)
                M *= p
            want.append(x - M if 2 * x > M else x)
        assert modular.crt(edge, bits=31 * K) == want


def test_plan_bounds_hold():
    rng = random.Random(13)
    tight = 0
    for f, g in _pairs(14, 60):
        pl = modular.plan(f, g)
        R = exact.resultant_y(f, g)
        if pl["zero"]:
            assert R == []
            continue
        assert len(R) - 1 <= pl["D"]
        assert all(abs(c) <= 1 << pl["bits"] for c in R)
        assert 30 * pl["nprimes"] >= pl["bits"] + 2
        tight += len(R) - 1 == pl["D"]
    assert tight >= 10  # the degree bound is reached by generic pairs
    del rng


def test_batch_is_thread_count_independent():
    pairs = _pairs(15, 20, dmax=7)
    assert modular.resultants(pairs, threads=1) == modular.resultants(pairs, threads=8)
    # chunking by the residue budget changes nothing
    assert modular.resultants(pairs, threads=3, max_words=1000) == modular.resultants(pairs, threads=3)


def test_digest_is_canonical():
    assert modular.digest([1, -2, 0]) == modular.digest([1, -2])
    assert modular.digest([]) != modular.digest([0, 1])
    assert modular.digest([255]) != modular.digest([-255])


# --------------------------------------------------------- planted mistakes

@pytest.mark.parametrize("plant", range(1, 8))
def test_planted_mistakes_are_caught(tmp_path, plant):
    """O2 compiled with one planted mistake (1 Euclid sign, 2 leading-coefficient
    power, 3 Lagrange sign, 4 no symmetric range, 5 g-rows first, 6 degree
    bound one too small, 7 sign-blind coefficient reduction) must fail the pins."""
    lib = modular.load(modular.build(target=str(tmp_path / f"libmodres_plant{plant}.so"),
                                     defines=[f"O2_PLANT={plant}"]))
    pairs = _pin_set(random.Random(16))
    want = [exact.resultant_y(f, g) for f, g in pairs]
    try:
        got = modular.resultants(pairs, threads=2, lib=lib)
    except RuntimeError:
        return  # the bound check refused a value: caught
    assert got != want


def test_unplanted_build_passes_the_same_pins(tmp_path):
    lib = modular.load(modular.build(target=str(tmp_path / "libmodres_clean.so"), defines=["O2_PLANT=0"]))
    pairs = _pin_set(random.Random(16))
    assert modular.resultants(pairs, threads=2, lib=lib) == [exact.resultant_y(f, g) for f, g in pairs]


def test_generator_layout_and_nested_lists_agree():
    pairs = inputs.workload_batch(2, n=3, deg_lo=2, deg_hi=4)
    a = modular.resultants(pairs)
    b = modular.resultants([(f.to_ints(), g.to_ints()) for f, g in pairs])
    c = modular.resultants([(np.asarray(f.coeffs), np.asarray(g.coeffs)) for f, g in pairs])
    assert a == b == c
