"""One modular image z_i^{(p)} = res(f(x_i, y), g(x_i, y), y) in Z_p
(Section 4.1) -- test infrastructure only.

The image is the determinant over Z_p of the Sylvester matrix of Section 3.1
with the formal y-degrees m_y, n_y of f and g kept, its Z[x] entries
evaluated at x_i and reduced mod p.  Since reduction mod p and evaluation at
x_i are ring homomorphisms Z[x] -> Z_p, this equals R^{(y)}(x_i) mod p for
every prime p and every point x_i.  The determinant is taken by plain
Gaussian elimination with row pivoting (numpy int64; p < 2^31 so every
product fits).
"""
import numpy as np

from .exact import sylvester, y_coefficients


def det_mod_p(M, p):
    """det(M) mod p for a square integer matrix (entries reduced first)."""
    A = np.array([[int(e) % p for e in row] for row in M], dtype=np.int64).reshape(len(M), len(M))
    n = A.shape[0]
    det = 1
    for k in range(n):
        nz = np.nonzero(A[k:, k])[0]
        if nz.size == 0:
            return 0
        piv = k + int(nz[0])
        if piv != k:
            A[[k, piv]] = A[[piv, k]]
            det = -det
        akk = int(A[k, k])
        det = det * akk % p
        inv = pow(akk, p - 2, p)
        if k + 1 < n:
            factors = (A[k + 1:, k] * inv) % p
            A[k + 1:, k:] = (A[k + 1:, k:] - (factors[:, None] * A[k, k:][None, :]) % p) % p
    return det % p


def eval_zx_mod(a, x0, p):
    v = 0
    for c in reversed(a):
        v = (v * x0 + c) % p
    return v


def resultant_image(f, g, p, x0):
    """det S^{(y)}(f, g)(x0) mod p, with f, g as in ``oracle.exact``."""
    fy, gy = y_coefficients(f), y_coefficients(g)
    if not fy or not gy:
        return 0
    S = sylvester(fy, gy)
    M = [[eval_zx_mod(e, x0, p) for e in row] for row in S]
    if not M:
        return 1 % p
    return det_mod_p(M, p)


def poly_eval_mod(coeffs, x0, p):
    """Value at x0 mod p of an integer polynomial given low-to-high."""
    return eval_zx_mod([int(c) for c in coeffs], x0, p)
