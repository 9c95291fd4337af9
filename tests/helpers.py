"""Shared helpers of the test-suite (test infrastructure, not product code)."""
import glob
import os
import random

from oracle import exact, modp
from oracle.exact import zx_add, zx_mul, zx_trim

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


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


def golden_var(path):
    """'y' for Res_y fixtures, 'x' for files with a `var: x` line."""
    for line in open(path):
        line = line.split("#")[0].strip()
        if line.startswith("var:"):
            return line.split(":")[1].strip()
    return "y"


def load_golden(path):
    f, g, R = {}, {}, {}
    for line in open(path):
        line = line.split("#")[0].strip()
        if not line or line.startswith("var:"):
            continue
        tag, rest = line.split(":")
        nums = [int(t) for t in rest.split()]
        if tag == "R":
            R[nums[0]] = nums[1]
        else:
            (f if tag == "f" else g)[(nums[0], nums[1])] = nums[2]

    def dense(d):
        nx = max(i for i, _ in d) + 1
        ny = max(j for _, j in d) + 1
        rows = [[0] * ny for _ in range(nx)]
        for (i, j), c in d.items():
            rows[i][j] = c
        return rows

    deg = max(R) if R else -1
    return dense(f), dense(g), zx_trim([R.get(k, 0) for k in range(deg + 1)])


ALL_GOLDEN = sorted(glob.glob(os.path.join(GOLDEN_DIR, "*.txt")))
GOLDEN = [p for p in ALL_GOLDEN if golden_var(p) == "y"]
GOLDEN_X = [p for p in ALL_GOLDEN if golden_var(p) == "x"]


def subst_y(g, alpha):
    """g(x, alpha(x)) in Z[x]."""
    gy = exact.y_coefficients(g)
    out, powa = [], [1]
    for gj in gy:
        out = zx_add(out, zx_mul(gj, powa))
        powa = zx_mul(powa, alpha)
    return out


def from_factors(a, alphas):
    """a(x) * prod (y - alpha_i(x)) as a dense f[i][j]."""
    poly = [list(a)]  # list over y-degree of Z[x] polys
    for al in alphas:
        nxt = [[] for _ in range(len(poly) + 1)]
        for j, c in enumerate(poly):
            nxt[j + 1] = zx_add(nxt[j + 1], c)
            nxt[j] = zx_add(nxt[j], zx_mul(c, [-t for t in al]))
        poly = nxt
    nx = max(len(c) for c in poly)
    return [[(poly[j][i] if i < len(poly[j]) else 0) for j in range(len(poly))] for i in range(nx)]


# ------------------------------------------------- full-size expected values

_FULL = {}


def full_size_records(name):
    """Expected (degree, bits, SHA-256) of every instance of a full-size
    workload, written by tests/golden/make_full_size.py from the oracle O2."""
    import json
    if not _FULL:
        _FULL.update(json.load(open(os.path.join(GOLDEN_DIR, "full_size.json")))["workloads"])
    return _FULL[name]["results"]


def assert_full_size(name, results, pairs=None, offset=0):
    """Every coefficient of every result equals the oracle's: the digest of
    the exact coefficient list must match the stored one.  On a mismatch the
    first failing instance is recomputed with O2 (when ``pairs`` is given)
    to name the first differing coefficient."""
    from oracle import modular
    recs = full_size_records(name)[offset:offset + len(results)]
    assert len(recs) == len(results), f"{name}: {len(results)} results, {len(recs)} expected values"
    bad = [i for i, (R, rec) in enumerate(zip(results, recs)) if modular.digest(R) != rec["sha256"]]
    if bad and pairs is not None:
        i = bad[0]
        want = modular.resultant(*pairs[i])
        got = results[i]
        first = next((k for k in range(max(len(want), len(got)))
                      if (want[k] if k < len(want) else 0) != (got[k] if k < len(got) else 0)), None)
        raise AssertionError(f"{name}: {len(bad)} of {len(results)} differ; instance {offset + i}: "
                             f"degree {len(got) - 1} vs {len(want) - 1}, first differing coefficient {first}")
    assert not bad, f"{name}: instances {[offset + i for i in bad[:10]]} differ from the oracle"
