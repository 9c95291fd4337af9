"""Parity of the tensor-core interpolation form (rs_config.g2_form = 4).

For one prime, the interpolation convolutions of every pair of a batch are
one exact matrix product on the tensor cores: residues split into bf16
digits, fp32 accumulation over 64 inputs at a time, and the digit-weight
classes recombined modulo p.  Here it is compared with the direct form and
with the oracles: small pairs coefficient by coefficient against O1, and the
whole 512-pair batch against O2's stored digests.  The row tiles are
exercised at their edges: one pair alone (2 of 128 rows), more than 64 pairs
of a prime (several tiles), point-pair counts M = 1 and M just above and
below multiples of 64.  Expected values never come from the GPU.
"""
import random

import pytest

from oracle import exact
from paper_1010_1386_gb300 import inputs, rs
from tests.helpers import assert_full_size, check_sampled_31, rand_bipoly

pytestmark = pytest.mark.gpu

TENSOR, DIRECT = 4, 1


@pytest.fixture(scope="module")
def tctx():
    c = rs.Context(device=0, timing=True, g2_form=TENSOR)
    yield c
    c.close()


def test_small_pairs_exact(tctx):
    rng = random.Random(41)
    pairs = []
    for _ in range(80):
        f = rand_bipoly(rng, rng.randint(0, 5), rng.randint(0, 6), bits=rng.choice([4, 20, 40, 90]))
        g = rand_bipoly(rng, rng.randint(0, 5), rng.randint(0, 6), bits=rng.choice([4, 20, 40, 90]))
        pairs.append((f, g))
    got = tctx.resultant_batch(pairs)
    for (f, g), R in zip(pairs, got):
        assert R == exact.resultant_y(f, g)
    for f, g in pairs[:4]:  # one pair alone: a row tile with 2 of its 128 rows
        assert tctx.resultant_y(f, g) == exact.resultant_y(f, g)


def test_same_as_direct_form_at_tile_edges():
    """Point-pair counts around multiples of 64 (tile lengths), M = 1, and
    more than 64 pairs sharing every prime (several row tiles per prime):
    the tensor form and the direct form give the same resultants bit for
    bit; a sample against the oracle."""
    rng = random.Random(42)
    pairs = []
    for dx, dy in [(0, 1), (1, 1), (1, 2), (3, 10), (4, 16), (8, 8), (7, 9), (16, 16), (2, 63), (1, 64),
                   (32, 2), (24, 40), (40, 40)]:
        bits = rng.choice([8, 31, 64])
        pairs.append((rand_bipoly(rng, dx, dy, bits=bits), rand_bipoly(rng, dx, dy, bits=bits)))
    for _ in range(150):  # many pairs of equal shape: 2+ full row tiles for each prime
        pairs.append((rand_bipoly(rng, 4, 8, bits=32), rand_bipoly(rng, 4, 8, bits=32)))
    got = {}
    for form in (DIRECT, TENSOR):
        with rs.Context(device=0, g2_form=form) as c:
            got[form] = c.resultant_batch(pairs)
    assert got[TENSOR] == got[DIRECT]
    for (f, g), R in list(zip(pairs, got[TENSOR]))[:6]:
        assert R == exact.resultant_y(f, g)
    rng2 = random.Random(43)
    for (f, g), R in list(zip(pairs, got[TENSOR]))[6:13]:
        check_sampled_31(f, g, R, rng2, samples=1)


def test_batch_full_size_exact(tctx):
    """All 512 pairs of the batched workload in one batch through the
    tensor-core form: every coefficient against the oracle O2's digests."""
    pairs = inputs.workload_batch(2, n=512)
    got = tctx.resultant_batch(pairs)
    assert_full_size("c2_batch", got, pairs)


def test_projections_full_size_exact():
    """Both projections of the dense degree-15 shift workload at k = 512
    (long point sequences, few pairs per prime) through the tensor form."""
    base = inputs.workload_shift(5, 15, False, 512)
    pairs = base + [(inputs.swap_xy(f), inputs.swap_xy(g)) for f, g in base]
    with rs.Context(device=0, g2_form=TENSOR) as c:
        got = c.resultant_batch(pairs)
    assert_full_size("shift_15_dense_512", got, pairs)
