"""Seeded synthetic inputs shaped like the resultant workloads.

This module only draws and lays out integer bivariate polynomials; it holds
none of the resultant arithmetic, so both the CUDA path and the CPU oracle
may consume what it produces.

Layout (the C ABI's, Eq. (2.1) notation): a polynomial f = sum f_ij x^i y^j
is a ``BiPoly`` whose ``coeffs`` is a uint32 array of shape
``(deg_x + 1, deg_y + 1, limbs)``; ``coeffs[i, j]`` holds f_ij as ``limbs``
little-endian 32-bit limbs in two's complement.
"""
from dataclasses import dataclass

import numpy as np


@dataclass
class BiPoly:
    coeffs: np.ndarray  # uint32 [deg_x+1][deg_y+1][limbs]

    @property
    def deg_x(self):
        return self.coeffs.shape[0] - 1

    @property
    def deg_y(self):
        return self.coeffs.shape[1] - 1

    @property
    def limbs(self):
        return self.coeffs.shape[2]

    def to_ints(self):
        """Nested list f[i][j] of Python ints."""
        c = self.coeffs
        L = c.shape[2]
        flat = c.reshape(-1, L)
        vals = [int.from_bytes(row.astype("<u4").tobytes(), "little", signed=True) for row in flat]
        nx, ny = c.shape[0], c.shape[1]
        return [vals[i * ny:(i + 1) * ny] for i in range(nx)]

    @staticmethod
    def from_ints(rows, limbs=None):
        nx = len(rows)
        ny = max((len(r) for r in rows), default=0)
        nx, ny = max(nx, 1), max(ny, 1)
        vals = [[(rows[i][j] if i < len(rows) and j < len(rows[i]) else 0) for j in range(ny)]
                for i in range(nx)]
        need = max((int(v).bit_length() + 1 for r in vals for v in r), default=1)
        L = max(1, -(-need // 32)) if limbs is None else limbs
        out = np.zeros((nx, ny, L), dtype=np.uint32)
        for i in range(nx):
            for j in range(ny):
                v = int(vals[i][j])
                if v:
                    b = v.to_bytes(4 * L, "little", signed=True)
                    out[i, j] = np.frombuffer(b, dtype="<u4")
        return BiPoly(out)


def swap_xy(f):
    """The same polynomial with x and y exchanged (a layout change only)."""
    return BiPoly(np.ascontiguousarray(f.coeffs.transpose(1, 0, 2)))


def signed_uniform_limbs(rng, shape, bits, limbs):
    """Uniform integers in [-2^(bits-1), 2^(bits-1)) as two's-complement
    limbs, shape ``shape + (limbs,)``; needs limbs * 32 >= bits."""
    assert limbs * 32 >= bits >= 2
    n = int(np.prod(shape)) if shape else 1
    nl = -(-bits // 32)
    u = rng.integers(0, 1 << 32, size=(n, nl), dtype=np.uint64).astype(np.uint32)
    top = bits - 32 * (nl - 1)  # bits used in the top drawn limb, 1..32
    if top < 32:
        u[:, nl - 1] &= np.uint32((1 << top) - 1)
    # u uniform in [0, 2^bits); u - 2^(bits-1) = flip bit bits-1 and sign-extend
    sb = np.uint32(1 << (top - 1))
    u[:, nl - 1] ^= sb
    neg = (u[:, nl - 1] & sb) != 0
    if top < 32:
        u[neg, nl - 1] |= np.uint32(((1 << 32) - 1) ^ ((1 << top) - 1))
    out = np.zeros((n, limbs), dtype=np.uint32)
    out[:, :nl] = u
    out[neg, nl:] = np.uint32(0xFFFFFFFF)
    return out.reshape(tuple(shape) + (limbs,))


def _nonzero_at(poly, i, j):
    if not poly.coeffs[i, j].any():
        poly.coeffs[i, j] = 0
        poly.coeffs[i, j, 0] = 1


def dense_total_degree(rng, deg, bits, limbs=None):
    """Dense f with all monomials x^i y^j, i + j <= deg, coefficients uniform
    signed ``bits``-bit; x^deg and y^deg made non-zero so the degrees hold."""
    L = limbs or -(-bits // 32)
    c = signed_uniform_limbs(rng, (deg + 1, deg + 1), bits, L)
    i = np.arange(deg + 1)[:, None]
    j = np.arange(deg + 1)[None, :]
    c[(i + j) > deg] = 0
    p = BiPoly(c)
    _nonzero_at(p, 0, deg)
    _nonzero_at(p, deg, 0)
    return p


def dense_bidegree(rng, deg_x, deg_y, bits, limbs=None):
    """Dense f with all monomials x^i y^j, i <= deg_x, j <= deg_y; the corner
    x^deg_x y^deg_y made non-zero so both degrees hold."""
    L = limbs or -(-bits // 32)
    p = BiPoly(signed_uniform_limbs(rng, (deg_x + 1, deg_y + 1), bits, L))
    _nonzero_at(p, deg_x, deg_y)
    return p


def small_uniform(rng, deg, lo, hi):
    """Dense total-degree polynomial with coefficients uniform in [lo, hi]."""
    v = rng.integers(lo, hi + 1, size=(deg + 1, deg + 1), dtype=np.int64)
    i = np.arange(deg + 1)[:, None]
    j = np.arange(deg + 1)[None, :]
    v[(i + j) > deg] = 0
    if v[0, deg] == 0:
        v[0, deg] = 1
    if v[deg, 0] == 0:
        v[deg, 0] = 1
    return BiPoly.from_ints(v.tolist(), limbs=1)


# ------------------------------------------------------------ workloads


def workload_small(seed=0):
    """One pair, dense total degree 6, coefficients uniform in [-2^10, 2^10]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [(small_uniform(rng, 6, -1024, 1024), small_uniform(rng, 6, -1024, 1024))]


def workload_single(seed=1, deg=30):
    """One pair, dense total degree 30, signed 32-bit uniform coefficients."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [(dense_total_degree(rng, deg, 32), dense_total_degree(rng, deg, 32))]


def workload_batch(seed=2, n=512, deg_lo=8, deg_hi=40, bit_choices=(16, 32, 64)):
    """n pairs; per pair one (deg_x, deg_y) drawn uniform in [deg_lo, deg_hi]
    and one bit length from ``bit_choices``, shared by f and g; bidegree-dense."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pairs = []
    for _ in range(n):
        dx = int(rng.integers(deg_lo, deg_hi + 1))
        dy = int(rng.integers(deg_lo, deg_hi + 1))
        b = int(rng.choice(bit_choices))
        pairs.append((dense_bidegree(rng, dx, dy, b), dense_bidegree(rng, dx, dy, b)))
    return pairs


def _ints_dense_total(rng, deg, bits):
    return dense_total_degree(rng, deg, bits).to_ints()


def _mul_dict(a, b):
    out = {}
    for (i1, j1), c1 in a.items():
        for (i2, j2), c2 in b.items():
            k = (i1 + i2, j1 + j2)
            out[k] = out.get(k, 0) + c1 * c2
    return {k: v for k, v in out.items() if v}


def _to_dict(rows):
    return {(i, j): c for i, r in enumerate(rows) for j, c in enumerate(r) if c}


def _from_dict(d):
    nx = max(i for i, _ in d) + 1
    ny = max(j for _, j in d) + 1
    rows = [[0] * ny for _ in range(nx)]
    for (i, j), c in d.items():
        rows[i][j] = c
    return rows


def _dy(d):
    return {(i, j - 1): j * c for (i, j), c in d.items() if j > 0}


def workload_nongeneric(seed=3, n=32, deg_p=24, deg_q=12, bits=64, coprime=False):
    """Topology-style non-generic pairs: f = p q^2 with p, q dense random
    (total degrees deg_p, deg_q), g = d f / d y (``coprime=False``: q divides
    both, so Res_y = 0) or g = d (p q) / d y (``coprime=True``)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pairs = []
    for _ in range(n):
        p = _to_dict(_ints_dense_total(rng, deg_p, bits))
        q = _to_dict(_ints_dense_total(rng, deg_q, bits))
        pq = _mul_dict(p, q)
        f = _mul_dict(pq, q)
        g = _dy(pq) if coprime else _dy(f)
        pairs.append((BiPoly.from_ints(_from_dict(f)), BiPoly.from_ints(_from_dict(g))))
    return pairs


def workload_serving(seed=4, n=10000, deg_lo=8, deg_hi=64, bits_lo=16, bits_hi=128):
    """Request stream: per request independent total degrees for f and g
    uniform in [deg_lo, deg_hi], one bit length uniform in [bits_lo, bits_hi],
    total-degree-dense.  Returns (pairs, unit-rate exponential gaps); scale the
    gaps by 1/rate for a Poisson stream of that rate."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pairs = []
    for _ in range(n):
        df = int(rng.integers(deg_lo, deg_hi + 1))
        dg = int(rng.integers(deg_lo, deg_hi + 1))
        b = int(rng.integers(bits_lo, bits_hi + 1))
        L = -(-b // 32)
        pairs.append((dense_total_degree(rng, df, b, L), dense_total_degree(rng, dg, b, L)))
    gaps = rng.exponential(1.0, size=n)
    return pairs, gaps


def workload_shift(seed=5, deg=9, sparse=False, k=128, curves=5):
    """The random-curve experiment with shifted coefficients: ``curves``
    random curves of total degree ``deg`` (dense: every monomial x^i y^j with
    i + j <= deg; sparse: each kept with probability 1/4, the x^deg and y^deg
    terms always), coefficients uniform signed 16-bit; each curve multiplied
    by 2^k with its constant coefficient raised by one.  Returns all
    curves * (curves - 1) / 2 pairs."""
    rng = np.random.Generator(np.random.PCG64(seed))
    polys = []
    for _ in range(curves):
        v = rng.integers(-(1 << 15), 1 << 15, size=(deg + 1, deg + 1), dtype=np.int64)
        i = np.arange(deg + 1)[:, None]
        j = np.arange(deg + 1)[None, :]
        v[(i + j) > deg] = 0
        if sparse:
            v[rng.random(size=v.shape) >= 0.25] = 0
        for a, b in ((0, deg), (deg, 0)):
            if v[a, b] == 0:
                v[a, b] = 1
        rows = [[int(c) << k for c in r] for r in v.tolist()]
        rows[0][0] += 1
        polys.append(BiPoly.from_ints(rows))
    return [(polys[a], polys[b]) for a in range(curves) for b in range(a + 1, curves)]

