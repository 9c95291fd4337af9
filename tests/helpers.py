"""Shared helpers of the test-suite (test infrastructure, not product code)."""
import random

from oracle import exact, modp


def rand_bipoly(rng, dx, dy, bits=20, density=1.0):
    """Dense-ish f[i][j] with signed coefficients of about ``bits`` bits and a
    non-zero corner x^dx y^dy."""
    b = 1 << (bits - 1)
    f = [[(rng.randint(-b, b - 1) if rng.random() < density else 0) for _ in range(dy + 1)]
         for _ in range(dx + 1)]
    if f[dx][dy] == 0:
        f[dx][dy] = 1
    return f


def eval_mod(R, x0, p):
    v = 0
    for c in reversed(R):
        v = (v * x0 + c) % p
    return v


def check_sampled(f, g, R, rng, samples=3, primes=(4294967291, 2305843009213693951, 1000000007)):
    """R(x0) = det S(x0) mod q for random q-sized points, q a prime unrelated
    to the library's table; exact R(0) and R(1) on tiny-enough inputs."""
    for q in primes[:samples]:
        x0 = rng.randrange(q)
        want = modp.resultant_image(f, g, q, x0) if q < (1 << 31) else None
        if want is None:
            continue
        assert eval_mod(R, x0, q) == want, f"R({x0}) mod {q} differs"


def check_sampled_31(f, g, R, rng, samples=2):
    """Random points modulo primes below 2^31 that are not in the library's
    table (the table holds primes in (2^31 - 2^20, 2^31))."""
    for q in (1000000007, 998244353, 2013265921)[:samples]:
        x0 = rng.randrange(q)
        assert eval_mod(R, x0, q) == modp.resultant_image(f, g, q, x0), f"R(x0) mod {q} differs"


def exact_points(f, g, R, points=(0, 1, -1)):
    for x0 in points:
        assert exact.zx_eval(R, x0) == exact.resultant_y_at(f, g, x0), f"R({x0}) differs"


def coprime_rng(seed):
    return random.Random(seed)
