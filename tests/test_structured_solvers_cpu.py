"""CPU models of the recurrences behind the two comparison variants (the
Schur recursion on the displacement generators of the Sylvester matrix, and
the two-stage triangular solve of the Vandermonde system on fractions, each
in the order of operations the CUDA kernels use), checked against the
oracle: the determinant of the Sylvester matrix mod p, and direct evaluation
of the interpolated polynomial.  They pin the derivations the kernels
follow; the GPU tests then compare the kernels with the default path and the
oracle bit for bit."""
import random

from oracle import modp

P = 2147483647  # the first prime of the library's table


def sylvester_mod(f, g, p):
    """S of Section 3.1 for f, g given by descending coefficient lists."""
    m, n = len(f) - 1, len(g) - 1
    r = m + n
    S = [[0] * r for _ in range(r)]
    for i in range(n):
        for k in range(m + 1):
            S[i][i + k] = f[k] % p
    for i in range(m):
        for k in range(n + 1):
            S[n + i][i + k] = g[k] % p
    return S


def schur_det(f, g, p, flip_sign=False):
    """det S mod p by the generalised Schur algorithm on the generators of
    M = S^T (M - Z M A^T = G B^T, A = Z_n (+) Z_m); None on a zero pivot."""
    m, n = len(f) - 1, len(g) - 1
    r = m + n
    G0 = [f[k] % p if k <= m else 0 for k in range(r)]
    G1 = [g[k] % p if k <= n else 0 for k in range(r)]
    B0 = [1 if k == 0 else 0 for k in range(r)]
    B1 = [1 if k == n else 0 for k in range(r)]
    num = den = c = 1
    for k in range(r):
        a, b, cc, d = G0[k], G1[k], B0[k], B1[k]
        t = (a * cc + b * d) % p
        if t == 0:
            return None
        num, den, c = num * t % p, den * c % p, c * t % p
        L = [(cc * G0[i] + d * G1[i]) % p for i in range(r)]
        G1 = [((b if flip_sign else -b) * G0[i] + a * G1[i]) % p for i in range(r)]
        U = [(a * B0[i] + b * B1[i]) % p for i in range(r)]
        B1 = [(-d * B0[i] + cc * B1[i]) % p for i in range(r)]
        G0 = [L[i - 1] if i >= 1 else 0 for i in range(r)]
        B0 = [U[i - 1] if i >= 1 and i != n else 0 for i in range(r)]
        assert all(G0[i] == G1[i] == B0[i] == B1[i] == 0 for i in range(k + 1))
    return num * pow(den, p - 2, p) % p


def test_schur_recursion_equals_sylvester_determinant():
    rng = random.Random(41)
    done = 0
    for _ in range(400):
        m, n = rng.randint(1, 8), rng.randint(1, 8)
        f = [rng.randrange(1, P)] + [rng.randrange(P) for _ in range(m)]
        g = [rng.randrange(1, P)] + [rng.randrange(P) for _ in range(n)]
        got = schur_det(f, g, P)
        if got is None:
            continue
        assert got == modp.det_mod_p(sylvester_mod(f, g, P), P)
        done += 1
    assert done > 390  # zero pivots are rare for random residues


def test_schur_breakdown_only_where_a_leading_minor_vanishes():
    # lc f = 0 (the formal degree kept): the first pivot vanishes
    assert schur_det([0, 3, 1], [1, 2], P) is None
    # a common root: det = 0, and the recursion cannot finish
    assert schur_det([1, -3, 2], [1, -1], P) is None  # (y-1)(y-2), y-1


def test_planted_sign_error_is_caught():
    """With the sign of the G_1 update flipped, the eliminated rows no
    longer vanish (the model's invariant) or the determinant is wrong."""
    rng = random.Random(42)
    caught = 0
    for _ in range(50):
        f = [rng.randrange(1, P) for _ in range(4)]
        g = [rng.randrange(1, P) for _ in range(3)]
        try:
            got = schur_det(f, g, P, flip_sign=True)
        except AssertionError:
            caught += 1
            continue
        caught += got is not None and got != modp.det_mod_p(sylvester_mod(f, g, P), P)
    assert caught > 45


def triangular_solve(xs, num, den, p, threads):
    """Coefficients c with sum_i c_i x_j^i = num_j / den_j: divided differences
    on fractions, one inversion, Newton to monomial; contiguous ranges per
    thread with the one neighbour value read before each stage."""
    N = len(xs)
    A, B = list(num), list(den)
    E = (N + threads - 1) // threads
    ranges = [(min(t * E, N), min(t * E + E, N)) for t in range(threads)]
    for k in range(N - 1):
        edge = [(A[max(b0, k + 1) - 1], B[max(b0, k + 1) - 1]) if max(b0, k + 1) < e0 else None
                for b0, e0 in ranges]
        for (b0, e0), ed in zip(ranges, edge):
            lo = max(b0, k + 1)
            for j in range(e0 - 1, lo - 1, -1):
                am, bm = (A[j - 1], B[j - 1]) if j > lo else ed
                A[j], B[j] = ((A[j] * bm - am * B[j]) % p,
                              B[j] * bm % p * ((xs[j] - xs[j - k - 1]) % p) % p)
    c = [A[j] * pow(B[j], p - 2, p) % p for j in range(N)]
    for k in range(N - 2, -1, -1):
        edge = [c[min(e0, N - 1)] if max(b0, k) < min(e0, N - 1) else None for b0, e0 in ranges]
        for (b0, e0), nx in zip(ranges, edge):
            lo, hi = max(b0, k), min(e0, N - 1)
            for j in range(lo, hi):
                c[j] = (c[j] - xs[k] * (c[j + 1] if j + 1 < hi else nx)) % p
    return c


def test_triangular_vandermonde_solve_interpolates():
    rng = random.Random(43)
    for _ in range(60):
        N = rng.randint(1, 40)
        q = rng.randrange(2, P - 1)
        xs = [(-1) ** (j & 1) * pow(q, j >> 1, P) % P for j in range(N)]  # the library's point order
        if len(set(xs)) < N:
            continue
        coef = [rng.randrange(P) for _ in range(N)]
        vals = [modp.eval_zx_mod(coef, x, P) for x in xs]
        den = [rng.randrange(1, P) for _ in range(N)]
        num = [v * d % P for v, d in zip(vals, den)]
        assert triangular_solve(xs, num, den, P, rng.choice([1, 3, 8, 256])) == coef
