"""Parity of the tensor-core CRT (rs_config.crt_form = 2): digits and limbs.

Garner's mixed-radix digits of a block of 64 primes take the contribution of
every earlier digit as one exact product on the tensor cores (bf16 digits of
the earlier digits and of W, fp32 accumulation read out every 64 digits,
each column reduced modulo its own prime), then the block's own triangle on
the CUDA cores.  The limbs sum_k v_k P_k are a second exact product: the
signed digits against the balanced bytes of the prefix products, by units
of 256 byte columns, with the fp32 columns carry-saved between windows.
Compared with the CUDA-core CRT kernels bit for bit and with the oracles:
prime counts on both sides of the 64-prime block boundaries (one block
only, exactly 64, 65, 128, 129, several hundred), coefficient counts that
leave the last 128-coefficient tile ragged, several tiles with many primes,
and the dense degree-15 shift workload at k = 512 against O2's digests.
Expected values never come from the GPU.
"""
import random

import pytest

from oracle import exact
from paper_1010_1386_gb300 import inputs, rs
from tests.helpers import assert_full_size, check_sampled_31, rand_bipoly

pytestmark = pytest.mark.gpu

TENSOR, CUDA_CORES = 2, 1


def _pairs_over_prime_counts(rng):
    """Pairs whose prime counts K cover 1 .. several blocks of 64 (the
    planner's K grows with the coefficient bits)."""
    pairs, ks = [], set()
    for bits in (4, 40, 200, 420, 500, 600, 900, 1300, 2000, 4000):
        for dx, dy in ((1, 2), (3, 3), (2, 6)):
            f = rand_bipoly(rng, dx, dy, bits=bits)
            g = rand_bipoly(rng, dx, dy, bits=bits)
            pairs.append((f, g))
            ks.add(rs.result_bound(f, g)["primes"])
    return pairs, ks


def test_same_as_cuda_core_digits_across_block_boundaries():
    rng = random.Random(51)
    pairs, ks = _pairs_over_prime_counts(rng)
    assert min(ks) < 64 and max(ks) > 256 and any(64 < k < 128 for k in ks), sorted(ks)
    got = {}
    for form in (CUDA_CORES, TENSOR):
        with rs.Context(device=0, crt_form=form) as c:
            got[form] = c.resultant_batch(pairs)
    assert got[TENSOR] == got[CUDA_CORES]
    for (f, g), R in list(zip(pairs, got[TENSOR]))[:6]:
        assert R == exact.resultant_y(f, g)
    rng2 = random.Random(52)
    for (f, g), R in list(zip(pairs, got[TENSOR]))[6:]:
        check_sampled_31(f, g, R, rng2, samples=1)


def test_exact_prime_counts_at_block_edges():
    """Single pairs with K = 64, 65, 128 and 129 primes exactly (found by
    raising the coefficient bits of a fixed shape), against the oracle."""
    rng = random.Random(53)
    want = {64, 65, 128, 129}
    found = {}
    base_f = rand_bipoly(rng, 1, 2, bits=8)
    base_g = rand_bipoly(rng, 1, 2, bits=8)
    for bits in range(8, 4000):
        f = [[c << bits for c in row] for row in base_f]
        g = [[c + (1 << bits) for c in row] for row in base_g]
        k = rs.result_bound(f, g)["primes"]
        if k in want and k not in found:
            found[k] = (f, g)
        if len(found) == len(want):
            break
    assert set(found) == want, sorted(found)
    pairs = [found[k] for k in sorted(found)]
    with rs.Context(device=0, crt_form=TENSOR) as c:
        got = c.resultant_batch(pairs)
        single = [c.resultant_y(f, g) for f, g in pairs]
    for (f, g), R, R1 in zip(pairs, got, single):
        ref = exact.resultant_y(f, g)
        assert R == ref and R1 == ref


def test_shift_workload_full_size_exact():
    """Both projections of the dense degree-15 curves scaled by 2^512
    (about 500 primes per resultant, eight digit blocks) through the
    tensor-core digits: every coefficient against the oracle O2's digests."""
    base = inputs.workload_shift(5, 15, False, 512)
    pairs = base + [(inputs.swap_xy(f), inputs.swap_xy(g)) for f, g in base]
    with rs.Context(device=0, crt_form=TENSOR) as c:
        got = c.resultant_batch(pairs)
    assert_full_size("shift_15_dense_512", got, pairs)


def test_many_coefficient_tiles_and_limb_units():
    """Pairs with 129 to 289 coefficients (two or three 128-row tiles, the
    last ragged) and 235 to about 2,500 primes (up to 40 chunks: many
    carry-saved windows, up to 39 units of 64 limbs): the tensor-core CRT
    against the CUDA-core one, every coefficient, and sampled values against
    the oracle."""
    rng = random.Random(54)
    pairs = []
    for bits, dx, dy in ((900, 6, 11), (2500, 8, 8), (300, 12, 12), (3000, 10, 13)):
        pairs.append((rand_bipoly(rng, dx, dy, bits=bits), rand_bipoly(rng, dx, dy, bits=bits)))
    shapes = [rs.result_bound(f, g) for f, g in pairs]
    assert any(b["deg"] + 1 > 256 for b in shapes) and all(b["deg"] + 1 > 128 for b in shapes), shapes
    assert max(b["primes"] for b in shapes) > 2048, shapes
    got = {}
    for form in (CUDA_CORES, TENSOR):
        with rs.Context(device=0, crt_form=form) as c:
            got[form] = c.resultant_batch(pairs)
    assert got[TENSOR] == got[CUDA_CORES]
    rng2 = random.Random(55)
    for (f, g), R in zip(pairs, got[TENSOR]):
        check_sampled_31(f, g, R, rng2, samples=2)
