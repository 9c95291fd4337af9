"""The modular arithmetic every kernel uses (csrc/modarith.cuh: Montgomery
form with R = 2^32, lazy two-product reduction, Fermat inverse) compiled as
host code and checked against Python's integers on edge values (0, 1, 2,
p - 1, p - 2, (p - 1) / 2, values near 2^31 and 2^32 for the conversion) and
random ones, for primes at both ends of the range the header allows and in
the library's table."""
import os
import random
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_1010_1386_gb300", "csrc", "modarith.cuh")

HARNESS = r"""
#include <stdio.h>
#include "modarith.cuh"
int main(void) {
  unsigned p, a, b, c, d, e;
  while (scanf("%u %u %u %u %u %u", &p, &a, &b, &c, &d, &e) == 6) {
    const ModP m = make_modp(p);
    const uint32_t A = to_mont(a, m), B = to_mont(b, m), C = to_mont(c, m), D = to_mont(d, m);
    const uint32_t mul = from_mont(mmul(A, B, m), m);
    const uint32_t mul2 = from_mont(mmul2(A, B, C, D, m), m);
    const uint32_t ar = a % p, br = b % p;
    const uint32_t add = madd(ar, br, p), sub = msub(ar, br, p), neg = mneg(ar, p);
    const uint32_t inv = A ? from_mont(minv(A, m), m) : 0u;
    const uint32_t pw = from_mont(mpow(A, e, m), m);
    printf("%u %u %u %u %u %u %u %u\n", from_mont(A, m), mul, mul2, add, sub, neg, inv, pw);
  }
  return 0;
}
"""


def is_prime(n):
    if n < 2:
        return False
    for q in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
        if n % q == 0:
            return n == q
    d, s = n - 1, 0
    while d % 2 == 0:
        d, s = d // 2, s + 1
    for a in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37):
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def primes_near(x, step):
    while not is_prime(x):
        x += step
    return x


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("modarith")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    exe = d / "h"
    subprocess.run([cxx, "-O2", "-x", "c++", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)],
                   check=True)
    return str(exe)


def test_montgomery_arithmetic_matches_python(harness):
    rng = random.Random(51)
    primes = [2147483647,                                  # the first table prime, 2^31 - 1
              primes_near((1 << 31) - (1 << 20) + 1, 2),   # near the table's lower end
              primes_near((1 << 30) + 1, 2),               # the smallest the header allows
              primes_near(rng.randrange(1 << 30, 1 << 31) | 1, 2)]
    cases = []
    for p in primes:
        edge = [0, 1, 2, p - 1, p - 2, (p - 1) // 2, p, p + 1, (1 << 31) - 1, (1 << 32) - 1]
        vals = edge + [rng.randrange(1 << 32) for _ in range(40)]
        for _ in range(400):
            a, b, c, d = (rng.choice(vals) for _ in range(4))
            e = rng.choice([0, 1, 2, p - 2, p - 1, rng.randrange(1 << 32)])
            cases.append((p, a, b, c, d, e))
    out = subprocess.run([harness], input="\n".join(" ".join(map(str, c)) for c in cases), text=True,
                         capture_output=True, check=True).stdout.split("\n")
    for (p, a, b, c, d, e), line in zip(cases, out):
        got = list(map(int, line.split()))
        ar, br, cr, dr = a % p, b % p, c % p, d % p
        want = [ar, ar * br % p, (ar * br + cr * dr) % p, (ar + br) % p, (ar - br) % p, (-ar) % p,
                pow(ar, p - 2, p) if ar else 0, pow(ar, e, p) if e else 1]
        assert got == want, (p, a, b, c, d, e)
    assert len(out) >= len(cases)
