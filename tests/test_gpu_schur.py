"""The paper's own structured solvers, built as comparison variants: the
Schur variant of the univariate resultants (rs_config.univariate = 1: the
generalised Schur algorithm on displacement generators of the Sylvester
matrix, one warp per image, elimination fallback on zero pivots) and the
interpolation by the triangular factorisation of the Vandermonde system
(rs_config.g2_form = 3), against the oracle and against the default path:
every image and every resultant must agree bit for bit."""
import random

import pytest

from oracle import exact, modp
from paper_1010_1386_gb300 import inputs, rs
from tests.helpers import rand_bipoly

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def schur():
    c = rs.Context(device=0, timing=True, univariate="schur")
    yield c
    c.close()


@pytest.fixture(scope="module")
def prs():
    c = rs.Context(device=0, timing=True)
    yield c
    c.close()


def times_y_minus_x(p):
    out = [[0] * (len(p[0]) + 1) for _ in range(len(p) + 1)]
    for i, row in enumerate(p):
        for j, c in enumerate(row):
            out[i][j + 1] += c
            out[i + 1][j] -= c
    return out


def test_images_equal_remainder_sequence_and_oracle(schur, prs):
    rng = random.Random(31)
    for dx, dy, bits in [(4, 5, 20), (2, 9, 64), (7, 3, 120), (1, 1, 8)]:
        f = rand_bipoly(rng, dx, dy, bits=bits)
        g = rand_bipoly(rng, dx + 1, max(1, dy - 2), bits=bits)
        for npts in (33, 70):
            p1, x1, z1 = schur.images(f, g, 4, npts)
            p2, x2, z2 = prs.images(f, g, 4, npts)
            assert (p1 == p2).all() and (x1 == x2).all()
            assert (z1 == z2).all()
            for k in range(4):
                for i in (0, 1, npts - 1, rng.randrange(npts)):
                    assert int(z1[k, i]) == modp.resultant_image(f, g, int(p1[k]), int(x1[k, i]))


def test_random_small_pairs_exact(schur):
    rng = random.Random(32)
    pairs = []
    for _ in range(40):
        f = rand_bipoly(rng, rng.randint(0, 5), rng.randint(0, 6), bits=rng.choice([4, 20, 60]))
        g = rand_bipoly(rng, rng.randint(0, 5), rng.randint(0, 6), bits=rng.choice([4, 20, 60]))
        pairs.append((f, g))
    for (f, g), R in zip(pairs, schur.resultant_batch(pairs)):
        assert R == exact.resultant_y(f, g)


def test_golden_examples(schur):
    from tests.helpers import GOLDEN, load_golden
    for path in GOLDEN:
        f, g, R = load_golden(path)
        assert schur.resultant_y(f, g) == R


def test_conventions_common_factor_and_fallback(schur):
    zero = [[0, 0], [0, 0]]
    g = [[1, 2], [3, 4]]
    assert schur.resultant_y(zero, g) == []
    f0 = [[2], [3]]  # m_y = 0: R = f^{n_y}
    h = rand_bipoly(random.Random(33), 2, 3)
    assert schur.resultant_y(f0, h) == exact.resultant_y(f0, h)
    assert schur.resultant_y(h, f0) == exact.resultant_y(h, f0)
    # a common factor: every leading principal minor chain breaks down and
    # every image goes through the elimination fallback
    rng = random.Random(34)
    a, b = rand_bipoly(rng, 2, 2), rand_bipoly(rng, 1, 3)
    F, G = times_y_minus_x(a), times_y_minus_x(b)
    bt = schur.batch([(F, G)])
    bt.run()
    assert bt.results() == [[]]
    info = bt.info()
    assert info["degenerate_images"] == info["images"]
    bt.close()


def test_unlucky_points_go_through_the_fallback(schur):
    """lc_y f = (x - 1)(x - 3): the first pivot vanishes at x = q^0 = 1 for
    every prime, so those images are finished by elimination."""
    rng = random.Random(35)
    g = rand_bipoly(rng, 3, 4, bits=30)
    f = rand_bipoly(rng, 2, 3, bits=30)
    f[0][3], f[1][3], f[2][3] = 3, -4, 1
    assert schur.resultant_y(f, g) == exact.resultant_y(f, g)
    bt = schur.batch([(f, g)])
    bt.run()
    info = bt.info()
    K = rs.result_bound(f, g)["primes"]
    assert info["unlucky_points"] >= K and info["degenerate_images"] >= K
    bt.close()


def test_abnormal_sequences(schur):
    rng = random.Random(36)
    for _ in range(8):
        f = [[0] * 5 for _ in range(3)]
        f[0][4] = 1
        f[0][0], f[1][0], f[2][0] = rng.randint(-9, 9), rng.randint(-9, 9), 1
        g = [[0] * 3 for _ in range(2)]
        g[0][2], g[1][0], g[0][0] = 1, rng.randint(-9, 9), rng.randint(-9, 9)
        assert schur.resultant_y(f, g) == exact.resultant_y(f, g)
        assert schur.resultant_y(g, f) == exact.resultant_y(g, f)


def test_full_size_equal_remainder_sequence(schur, prs):
    [(f, g)] = inputs.workload_small(0)
    assert schur.resultant_y(f, g) == exact.resultant_y(f.to_ints(), g.to_ints())
    pairs = inputs.workload_batch(2, n=512)[:24]
    assert schur.resultant_batch(pairs) == prs.resultant_batch(pairs)


def test_largest_generators(schur, prs):
    """m_y + n_y = 142 (five rows per lane), and 33 (two slots, one row in
    the second)."""
    rng = random.Random(37)
    for dy_f, dy_g in [(71, 71), (17, 16)]:
        f = rand_bipoly(rng, 1, dy_f, bits=12)
        g = rand_bipoly(rng, 1, dy_g, bits=12)
        assert schur.resultant_y(f, g) == prs.resultant_y(f, g)


# ---------------------------------------- interpolation by triangular factorisation

@pytest.fixture(scope="module")
def tri():
    c = rs.Context(device=0, timing=True, g2_form=3)
    yield c
    c.close()


def test_triangular_interpolation_exact(tri):
    rng = random.Random(38)
    pairs = []
    for _ in range(30):
        f = rand_bipoly(rng, rng.randint(0, 5), rng.randint(0, 6), bits=rng.choice([4, 30, 70]))
        g = rand_bipoly(rng, rng.randint(0, 5), rng.randint(0, 6), bits=rng.choice([4, 30, 70]))
        pairs.append((f, g))
    for (f, g), R in zip(pairs, tri.resultant_batch(pairs)):
        assert R == exact.resultant_y(f, g)
    from tests.helpers import GOLDEN, load_golden
    for path in GOLDEN:
        f, g, R = load_golden(path)
        assert tri.resultant_y(f, g) == R


def test_triangular_interpolation_full_size(tri, prs):
    [(f, g)] = inputs.workload_single(1)  # D + 1 = 901 points, 76 primes
    assert tri.resultant_y(f, g) == prs.resultant_y(f, g)
    pairs = inputs.workload_batch(2, n=512)[:24]
    assert tri.resultant_batch(pairs) == prs.resultant_batch(pairs)


def test_paper_design_end_to_end(prs):
    """Both of the paper's structured solvers at once: Schur on the
    generators for the images and the triangular factorisation for the
    interpolation."""
    pairs = inputs.workload_batch(2, n=512)[:12] + inputs.workload_small(0)
    with rs.Context(device=0, univariate="schur", g2_form=3) as c:
        assert c.resultant_batch(pairs) == prs.resultant_batch(pairs)
