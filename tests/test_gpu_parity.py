"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Small inputs are compared coefficient by coefficient with the exact oracle
O1; every instance of the full-size workloads (the single dense degree-30
pair, all 512 pairs of the batch, all 32 pairs of the non-generic batch
f = p q^2, g = f_y and of its coprime variant, the first 512 requests of the
serving stream) is compared coefficient by coefficient with the
independent modular oracle O2 through the stored digests of its exact
results (tests/golden/full_size.json).  Sampled modular images are checked
against det S(x_i) mod p at the library's own points.  Expected values never
come from the GPU.
"""
import random

import numpy as np
import pytest

from oracle import exact, modp
from paper_1010_1386_gb300 import inputs, rs
from tests.helpers import assert_full_size, check_sampled_31, eval_mod, rand_bipoly

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = rs.Context(device=0, timing=True)
    yield c
    c.close()


def oracle(f, g):
    return exact.resultant_y(f, g)


# ----------------------------------------------------------- exact, small

def test_small_config_exact(ctx):
    [(f, g)] = inputs.workload_small(0)
    F, G = f.to_ints(), g.to_ints()
    assert ctx.resultant_y(f, g) == oracle(F, G)


def test_random_small_pairs_exact(ctx):
    rng = random.Random(1)
    pairs = []
    for _ in range(60):
        f = rand_bipoly(rng, rng.randint(0, 5), rng.randint(0, 6), bits=rng.choice([4, 20, 40, 90]))
        g = rand_bipoly(rng, rng.randint(0, 5), rng.randint(0, 6), bits=rng.choice([4, 20, 40, 90]))
        pairs.append((f, g))
    got = ctx.resultant_batch(pairs)
    for (f, g), r in zip(pairs, got):
        assert r == oracle(f, g)
    for f, g in pairs[:8]:
        assert ctx.resultant_y(f, g) == oracle(f, g)


def test_golden_examples(ctx):
    from tests.helpers import GOLDEN, load_golden
    for path in GOLDEN:
        f, g, R = load_golden(path)
        assert ctx.resultant_y(f, g) == R


def test_conventions_and_degenerate_inputs(ctx):
    zero = [[0, 0], [0, 0]]
    g = [[1, 2], [3, 4]]
    assert ctx.resultant_y(zero, g) == []
    assert ctx.resultant_y(g, zero) == []
    assert ctx.resultant_y([[5]], [[7], [1]]) == [1]
    f0 = [[2], [3]]  # m_y = 0: R = f^{n_y}
    h = rand_bipoly(random.Random(2), 2, 3)
    assert ctx.resultant_y(f0, h) == oracle(f0, h)
    assert ctx.resultant_y(h, f0) == oracle(h, f0)
    # common factor (y - x): R = 0, every image meets a zero pivot
    rng = random.Random(3)
    a, b = rand_bipoly(rng, 2, 2), rand_bipoly(rng, 1, 3)

    def times_y_minus_x(p):
        out = [[0] * (len(p[0]) + 1) for _ in range(len(p) + 1)]
        for i, row in enumerate(p):
            for j, c in enumerate(row):
                out[i][j + 1] += c
                out[i + 1][j] -= c
        return out
    assert ctx.resultant_y(times_y_minus_x(a), times_y_minus_x(b)) == []
    # zero rows / columns are trimmed
    padded = [row + [0, 0] for row in h] + [[0] * (len(h[0]) + 2)]
    assert ctx.resultant_y(padded, f0) == oracle(h, f0)


def test_unlucky_points_and_primes(ctx):
    """lc_y f vanishing at x = 1 (the first evaluation point +q^0 for every
    prime) and at x = 3, and a leading coefficient divisible by the first
    table prime 2^31 - 1."""
    rng = random.Random(4)
    g = rand_bipoly(rng, 3, 4, bits=30)
    # lc_y f = (x - 1)(x - 3) = x^2 - 4 x + 3
    f = rand_bipoly(rng, 2, 3, bits=30)
    f[0][3], f[1][3], f[2][3] = 3, -4, 1
    assert ctx.resultant_y(f, g) == oracle(f, g)
    primes, pts, imgs = ctx.images(f, g, 3, 8)
    for k in range(3):
        assert int(pts[k, 0]) == 1  # x = q^0 = 1: lc_y f vanishes there
        for i in range(8):
            assert int(imgs[k, i]) == modp.resultant_image(f, g, int(primes[k]), int(pts[k, i]))
    b = ctx.batch([(f, g)])
    b.run()
    info = b.info()
    assert info["unlucky_points"] >= rs.result_bound(f, g)["primes"]  # x = q^0 = 1, every prime
    b.close()
    f2 = rand_bipoly(rng, 2, 3, bits=30)
    f2[0][3], f2[1][3], f2[2][3] = 2147483647, 0, 0
    g2 = rand_bipoly(rng, 2, 3, bits=30)
    g2[0][3], g2[1][3], g2[2][3] = 3 * 2147483647, 0, 0
    assert ctx.resultant_y(f2, g2) == oracle(f2, g2)
    b = ctx.batch([(f2, g2)])
    b.run()
    assert b.info()["unlucky_primes"] >= 1
    b.close()


def test_abnormal_remainder_sequences(ctx):
    """Specialised pairs whose remainder sequences skip degrees (zero pivots)."""
    rng = random.Random(5)
    for _ in range(10):
        # f = y^4 + c(x): g's odd terms vanish -> sparse sequences
        f = [[0] * 5 for _ in range(3)]
        f[0][4] = 1
        f[0][0], f[1][0], f[2][0] = rng.randint(-9, 9), rng.randint(-9, 9), 1
        g = [[0] * 3 for _ in range(2)]
        g[0][2], g[1][0], g[0][0] = 1, rng.randint(-9, 9), rng.randint(-9, 9)
        assert ctx.resultant_y(f, g) == oracle(f, g)
        assert ctx.resultant_y(g, f) == oracle(g, f)


# ------------------------------------------------------------ modular images

def test_images_against_oracle(ctx):
    rng = random.Random(6)
    for dx, dy, bits in [(6, 6, 11), (3, 9, 64), (9, 2, 200)]:
        f = rand_bipoly(rng, dx, dy, bits=bits)
        g = rand_bipoly(rng, dx + 1, dy - 1 if dy > 1 else dy, bits=bits)
        for npts in (70, 71):  # an even and an odd number of points
            primes, pts, imgs = ctx.images(f, g, 5, npts)
            assert primes[0] == 2147483647 and all(primes[i] > primes[i + 1] for i in range(4))
            for k in range(5):
                p = int(primes[k])
                assert len(set(int(v) for v in pts[k])) == npts  # distinct points
                # pairs +-q^t: x_{2t+1} = -x_{2t}, x_{2t+2} = x_{2t} x_2
                assert int(pts[k, 0]) == 1
                assert all((int(pts[k, 2 * t]) + int(pts[k, 2 * t + 1])) % p == 0 for t in range(npts // 2))
                assert all(int(pts[k, 2 * t]) * int(pts[k, 2]) % p == int(pts[k, 2 * t + 2])
                           for t in range((npts - 1) // 2))
                for i in list(range(8)) + [npts - 1] + [rng.randrange(npts) for _ in range(6)]:
                    assert int(imgs[k, i]) == modp.resultant_image(f, g, p, int(pts[k, i]))


# ---------------------------------------------------------- full-size configs

def test_single_dense30_full_size(ctx):
    """The single pair of dense total degree 30 (signed 32-bit): every coefficient
    against the oracle O2, the planner's bounds, and sampled images against
    the result reduced at the library's own points."""
    [(f, g)] = inputs.workload_single(1)
    R = ctx.resultant_y(f, g)
    assert_full_size("c1_single", [R], [(f, g)])
    bound = rs.result_bound(f, g)
    assert len(R) - 1 <= bound["deg"] == 900
    assert max(abs(c) for c in R).bit_length() < bound["bits"]
    primes, pts, imgs = ctx.images(f, g, 3, 901)
    for k in range(3):
        for i in (0, 1, 450, 900):
            assert int(imgs[k, i]) == eval_mod(R, int(pts[k, i]), int(primes[k]))


def test_batch_full_size_exact(ctx):
    """The 512-pair batch, all pairs in one batch: every coefficient of every
    resultant against the oracle O2, and the degree bound."""
    pairs = inputs.workload_batch(2, n=512)
    got = ctx.resultant_batch(pairs)
    assert_full_size("c2_batch", got, pairs)
    for (f, g), R in zip(pairs, got):
        assert len(R) - 1 <= rs.result_bound(f, g)["deg"]


def test_nongeneric_literal_is_zero(ctx):
    """All 32 pairs of the literal topology workload at full size: q divides
    f and g, so every resultant is exactly zero (and every image degenerate)."""
    pairs = inputs.workload_nongeneric(3, n=32)
    with rs.Context(device=0, timing=True) as c:
        b = c.batch(pairs)
        b.run()
        got = b.results()
        info = b.info()
        b.close()
    assert all(R == [] for R in got)
    assert_full_size("c3_nongeneric", got, pairs)
    assert info["degenerate_images"] == info["images"]


def test_nongeneric_coprime_full_size(ctx):
    """The coprime topology workload at full size (f = p q^2, g = d(pq)/dy,
    total degrees 48 and 35, 64-bit coefficients): every coefficient of all
    32 resultants against the oracle O2, and for the first pair the exact
    identity Res_y(p q^2, g) = Res_y(p, g) Res_y(q, g)^2 from three GPU
    resultants."""
    pairs = inputs.workload_nongeneric(3, n=32, coprime=True)
    got = ctx.resultant_batch(pairs)
    assert_full_size("c3p_nongeneric_coprime", got, pairs)
    for (f, g), R in zip(pairs, got):
        b = rs.result_bound(f, g)
        assert len(R) - 1 <= b["deg"]
        assert R and max(abs(c) for c in R).bit_length() < b["bits"]
    # the generator's first draw, replayed: p and q of pair 0
    from paper_1010_1386_gb300.inputs import _dy, _from_dict, _mul_dict, _to_dict
    g0 = np.random.Generator(np.random.PCG64(3))
    p = inputs.dense_total_degree(g0, 24, 64).to_ints()
    q = inputs.dense_total_degree(g0, 12, 64).to_ints()
    PQ = _mul_dict(_to_dict(p), _to_dict(q))
    f0, gg = _from_dict(_mul_dict(PQ, _to_dict(q))), _from_dict(_dy(PQ))
    assert f0 == pairs[0][0].to_ints() and gg == pairs[0][1].to_ints()
    Rp, Rq = ctx.resultant_batch([(p, gg), (q, gg)])
    assert got[0] == exact.zx_mul(Rp, exact.zx_mul(Rq, Rq))


def test_serving_requests_batched_exact(ctx):
    """The first 512 requests of the serving stream (total degrees 8..64,
    16..128-bit coefficients) in one batch: every coefficient against the
    oracle O2."""
    pairs, _ = inputs.workload_serving(4, n=512)
    got = ctx.resultant_batch(pairs)
    assert_full_size("c4_serving_first512", got, pairs)


def test_nongeneric_coprime_multiplicative(ctx):
    """f = p q^2, g = d(pq)/dy: Res_y(f, g) = Res_y(p, g) Res_y(q, g)^2,
    checked exactly with three independent GPU resultants, plus sampled
    values against the oracle."""
    rng = np.random.Generator(np.random.PCG64(3))
    p = inputs.dense_total_degree(rng, 8, 64).to_ints()
    q = inputs.dense_total_degree(rng, 4, 64).to_ints()
    from paper_1010_1386_gb300.inputs import _dy, _from_dict, _mul_dict, _to_dict
    P, Q = _to_dict(p), _to_dict(q)
    PQ = _mul_dict(P, Q)
    f = _from_dict(_mul_dict(PQ, Q))
    g = _from_dict(_dy(PQ))
    Rf, Rp, Rq = ctx.resultant_batch([(f, g), (p, g), (q, g)])
    assert Rf == exact.zx_mul(Rp, exact.zx_mul(Rq, Rq))
    check_sampled_31(f, g, Rf, random.Random(9), samples=2)


def test_g2_transform_and_direct_forms_agree():
    """The interpolation stage by number-theoretic transforms (three NTT
    primes, exact integer convolutions) and by direct lazily reduced dot
    products give the same residues, so the same resultants bit for bit:
    point counts at and around transform-length boundaries (N = 2^k + 1 needs
    the next length), tiny degrees, and the batched workload's first pairs;
    small pairs also against the oracle."""
    rng = random.Random(17)
    pairs = []
    for dx, dy in [(0, 1), (1, 1), (1, 2), (2, 3), (8, 16), (16, 16), (16, 32), (1, 64), (24, 40), (40, 40)]:
        bits = rng.choice([8, 31, 64])
        pairs.append((rand_bipoly(rng, dx, dy, bits=bits), rand_bipoly(rng, dx, dy, bits=bits)))
    pairs += [(f.to_ints(), g.to_ints()) for f, g in inputs.workload_batch(2, n=512)[:24]]
    got = {}
    for form in (1, 2, 0):
        with rs.Context(device=0, g2_form=form) as c:
            got[form] = c.resultant_batch(pairs)
    assert got[1] == got[2] and got[0] == got[1]
    for (f, g), R in list(zip(pairs, got[2]))[:4]:
        assert R == oracle(f, g)
    rng2 = random.Random(18)
    for (f, g), R in list(zip(pairs, got[2]))[4:10]:
        check_sampled_31(f, g, R, rng2, samples=1)


def test_maximum_capacity_and_limbs(ctx):
    rng = random.Random(10)
    f = rand_bipoly(rng, 2, 71, bits=40)
    g = rand_bipoly(rng, 1, 70, bits=40)
    R = ctx.resultant_y(f, g)
    check_sampled_31(f, g, R, rng, samples=2)
    wide_f = rand_bipoly(rng, 2, 3, bits=4090)
    wide_g = rand_bipoly(rng, 3, 2, bits=4090)
    assert inputs.BiPoly.from_ints(wide_f).limbs == rs.RS_MAX_LIMBS
    assert ctx.resultant_y(wide_f, wide_g) == oracle(wide_f, wide_g)


def test_errors(ctx):
    rng = random.Random(11)
    with pytest.raises(rs.RsError) as e:
        ctx.resultant_y(rand_bipoly(rng, 1, 72), rand_bipoly(rng, 1, 2))
    assert e.value.code == -6
    lib = rs.load()
    P = rs._Polys([[[1, 2], [3, 4]], [[5, 1]]])
    out = (rs.rs_upoly * 1)()
    out[0].capacity_words = 0
    rc = lib.rs_resultant_y(ctx.h, P.structs, rs.ctypes.byref(P.structs[1]), out)
    assert rc == -2 and out[0].deg >= 0
    assert lib.rs_resultant_y(ctx.h, None, None, out) == -1


def test_batches_on_caller_streams_overlap_exactly(ctx):
    """rs_batch_create_on: two prepared batches on two caller streams,
    alternated with the result copy of one overlapping the other's run,
    give the same results as the context's own path, step after step."""
    torch = pytest.importorskip("torch")
    rng = random.Random(9)
    pairs = [(rand_bipoly(rng, rng.randint(1, 6), rng.randint(1, 6), bits=40),
              rand_bipoly(rng, rng.randint(1, 6), rng.randint(1, 6), bits=40)) for _ in range(24)]
    want = ctx.resultant_batch(pairs)
    streams = [torch.cuda.Stream(device=0) for _ in range(2)]
    bs = [ctx.batch(pairs, stream=st.cuda_stream) for st in streams]
    prev = None
    for s in range(5):
        b = bs[s % 2]
        b.upload(pairs)
        b.run()
        if prev is not None:
            assert prev.results() == want
        prev = b
    assert prev.results() == want
    for b in bs:
        b.close()


def test_product_formula_full_size(ctx):
    """Every coefficient of a large resultant against the closed form
    Res_y(f, g) = a^{n_y} prod_i g(x, alpha_i(x)) for f = a prod_{i<30}
    (y - alpha_i(x)) (plain Z[x] arithmetic, no determinant): m_y = 30,
    n_y = 20, deg R = 1000, coefficients of up to about 3,700 bits."""
    from oracle.exact import zx_mul, zx_trim
    from tests.helpers import from_factors, subst_y
    rng = random.Random(11)
    a = [rng.randint(-40, 40) for _ in range(3)]
    a[-1] = a[-1] or 7
    alphas = [[rng.randint(-40, 40), rng.randint(-40, 40) or 1] for _ in range(30)]
    f = from_factors(a, alphas)
    g = rand_bipoly(rng, 12, 20, bits=20)
    expect = [1]
    for _ in range(20):
        expect = zx_mul(expect, zx_trim(a))
    for al in alphas:
        expect = zx_mul(expect, subst_y(g, al))
    got = ctx.resultant_y(f, g)
    assert len(got) == 1001 and got == expect


def test_crt_one_thread_per_coefficient_small_prime_counts(ctx):
    """A batch with enough coefficients (about 170,000) to take the CRT digit
    kernel with one thread per coefficient, made of small pairs whose prime
    counts run from 1 to about 25 (groups of four digit rows, partial ones
    included): every result against the oracle O2, a sample against O1."""
    from oracle import modular
    rng = random.Random(71)
    pairs = []
    for i in range(4000):
        bits = 2 + (i % 12) * 6
        dx, dy = rng.randint(3, 6), rng.randint(3, 6)
        pairs.append((rand_bipoly(rng, dx, dy, bits=bits), rand_bipoly(rng, dx, dy, bits=bits)))
    nc = sum(rs.result_bound(f, g)["deg"] + 1 for f, g in pairs)
    ks = {rs.result_bound(f, g)["primes"] for f, g in pairs[:24]}
    assert nc >= 256 * 152 and {1, 2, 3, 5} <= ks, (nc, ks)
    got = ctx.resultant_batch(pairs)
    assert got == modular.resultants(pairs)
    for i in range(0, 4000, 500):
        assert got[i] == oracle(*pairs[i])
