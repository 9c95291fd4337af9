"""Both projections (Section 3.1): R^{(x)} = res(f, g, x) through
rs_resultant_x and the paired call rs_projections, against the oracle's own
x-resultant (exact on small inputs and the worked examples), and every
coefficient of both projections of the random-curve workload with
coefficients shifted by 2^k (up to ~2000 primes per resultant) against the
independent modular oracle O2."""
import random

import pytest

from oracle import exact
from paper_1010_1386_gb300 import inputs, rs
from tests.helpers import assert_full_size, rand_bipoly
from tests.helpers import GOLDEN_X, load_golden

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = rs.Context(device=0)
    yield c
    c.close()


def test_resultant_x_exact_small(ctx):
    for path in GOLDEN_X:
        f, g, R = load_golden(path)
        assert ctx.resultant_x(f, g) == R, path
    rng = random.Random(51)
    for _ in range(20):
        f = rand_bipoly(rng, rng.randint(0, 5), rng.randint(0, 5), bits=rng.choice([4, 30, 70]))
        g = rand_bipoly(rng, rng.randint(0, 5), rng.randint(0, 5), bits=rng.choice([4, 30, 70]))
        assert ctx.resultant_x(f, g) == exact.resultant_x(f, g)


def test_projections_match_single_calls_and_oracle(ctx):
    rng = random.Random(52)
    pairs = [(rand_bipoly(rng, rng.randint(1, 6), rng.randint(1, 6), bits=rng.choice([8, 40])),
              rand_bipoly(rng, rng.randint(1, 6), rng.randint(1, 6), bits=rng.choice([8, 40])))
             for _ in range(24)]
    Ry, Rx = ctx.projections(pairs)
    for (f, g), ry, rx in zip(pairs, Ry, Rx):
        assert ry == ctx.resultant_y(f, g)
        assert rx == ctx.resultant_x(f, g)
    for (f, g), ry, rx in list(zip(pairs, Ry, Rx))[:8]:
        assert ry == exact.resultant_y(f, g) and rx == exact.resultant_x(f, g)
    # a planted common root (x0, y0) = (3, -2) projects to roots of both
    f = [[5, 0, 1], [1, 1, 0]]             # 5 + y^2 + x + x y  -> at (3,-2): 5 + 4 + 3 - 6 = 6
    f[0][0] -= 6
    g = [[0, 2], [1, 0], [1, 0]]           # 2y + x + x^2 -> at (3,-2): -4 + 3 + 9 = 8
    g[0][0] -= 8
    (ry,), (rx,) = ctx.projections([(f, g)])
    assert exact.zx_eval(ry, 3) == 0 and exact.zx_eval(rx, -2) == 0


@pytest.mark.parametrize("deg,sparse,k", [(9, False, 128), (9, True, 2048), (15, False, 512), (15, False, 2048)])
def test_shift_workload_projections(ctx, deg, sparse, k):
    """All 10 pairs of five random curves scaled by 2^k (constant term + 1),
    up to about 2,000 primes per resultant: every coefficient of both
    projections against the oracle O2, and the planner's bounds."""
    pairs = inputs.workload_shift(5, deg, sparse, k)
    Ry, Rx = ctx.projections(pairs)
    name = f"shift_{deg}_{'sparse' if sparse else 'dense'}_{k}"
    swapped = [(inputs.swap_xy(f), inputs.swap_xy(g)) for f, g in pairs]
    assert_full_size(name, Ry, pairs)
    assert_full_size(name, Rx, swapped, offset=len(pairs))
    for (f, g), (fs, gs), ry, rx in zip(pairs, swapped, Ry, Rx):
        by, bx = rs.result_bound(f, g), rs.result_bound(fs, gs)
        assert len(ry) - 1 <= by["deg"] and max(abs(c) for c in ry).bit_length() < by["bits"]
        assert len(rx) - 1 <= bx["deg"] and max(abs(c) for c in rx).bit_length() < bx["bits"]
