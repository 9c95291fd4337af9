"""O2: the independent modular resultant (``oracle/modres.c``) -- TEST
INFRASTRUCTURE ONLY.

R^{(y)} = res(f, g, y) in Z[x] (Section 3.1) by the modular method of
Section 4.1 in its plainest form: this oracle's own primes (the largest below
2^31 - 2^20), consecutive integer points x = 0..D, one Sylvester determinant
mod p per (prime, point) by the Euclidean algorithm (or by Gaussian
elimination of the formal Sylvester matrix where a leading coefficient
vanishes at the point), Lagrange interpolation, and the constructive Chinese
remainder theorem on a small bignum.  It shares no code with the CUDA path
and no code with ``oracle.exact`` (O1), against which it is pinned in
``tests/test_oracle_modular.py``.

This module only marshals arguments and converts limbs; ``build()`` compiles
the C file with the host compiler (no GPU, no product code).  Only
``tests/``, ``__graft_entry__`` and the CPU legs of ``bench.py`` may use it.
"""
import ctypes
import hashlib
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "modres.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libmodres.so")
CC = os.environ.get("CC", "gcc")

O2_ERR = {-1: "bad argument", -2: "out of memory", -3: "a CRT value exceeds the coefficient bound",
          -4: "more primes than the table holds"}


class _Poly(ctypes.Structure):
    _fields_ = [("deg_x", ctypes.c_int32), ("deg_y", ctypes.c_int32), ("limbs", ctypes.c_int32),
                ("coeffs", ctypes.POINTER(ctypes.c_uint32))]


class _Plan(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in
                ("m_y", "n_y", "m_x", "n_x", "D", "bits", "nprimes", "out_limbs", "zero", "pad")]


def build(source=SRC, target=LIB, defines=()):
    """Compile the oracle's C file into a shared library if it is missing or
    older than its source.  ``defines`` (test use only) are passed as -D."""
    os.makedirs(os.path.dirname(target), exist_ok=True)
    if os.path.exists(target) and os.path.getmtime(target) >= os.path.getmtime(source) and not defines:
        return target
    tmp = target + ".tmp%d" % os.getpid()
    cmd = [CC, "-O2", "-std=c11", "-fPIC", "-shared", "-pthread"] + ["-D" + d for d in defines] + \
        [source, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("oracle build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    os.replace(tmp, target)
    return target


_libs = {}


def load(path=None):
    path = path or build()
    lib = _libs.get(path)
    if lib is None:
        lib = ctypes.CDLL(path)
        P = ctypes.POINTER(_Poly)
        lib.o2_plan_pair.argtypes = [P, P, ctypes.POINTER(_Plan)]
        lib.o2_resultant_batch.argtypes = [ctypes.c_int32, P, P, ctypes.c_int32,
                                           ctypes.POINTER(ctypes.POINTER(ctypes.c_uint32)),
                                           ctypes.POINTER(ctypes.c_int32)]
        lib.o2_image.restype = ctypes.c_uint32
        lib.o2_image.argtypes = [P, P, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_int32,
                                 ctypes.POINTER(ctypes.c_int32)]
        lib.o2_residues.argtypes = [P, P, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32)]
        lib.o2_crt.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(ctypes.c_uint32), ctypes.c_int32,
                               ctypes.c_int32, ctypes.POINTER(ctypes.c_uint32)]
        lib.o2_prime.restype = ctypes.c_uint32
        lib.o2_prime.argtypes = [ctypes.c_int32]
        _libs[path] = lib
    return lib


# ------------------------------------------------------------- marshalling

def limbs_array(f):
    """uint32 array [deg_x + 1][deg_y + 1][limbs] (two's complement) of a
    polynomial given as such an array, an object with ``.coeffs``, or a
    nested list f[i][j] of Python ints."""
    c = getattr(f, "coeffs", f)
    if isinstance(c, np.ndarray):
        return np.ascontiguousarray(c, dtype=np.uint32)
    rows = [list(r) for r in c] or [[0]]
    nx = len(rows)
    ny = max(1, max(len(r) for r in rows))
    vals = [int(rows[i][j]) if j < len(rows[i]) else 0 for i in range(nx) for j in range(ny)]
    need = max([(v if v >= 0 else ~v).bit_length() + 1 for v in vals] + [1])
    L = -(-need // 32)
    out = np.zeros((nx * ny, L), dtype=np.uint32)
    for k, v in enumerate(vals):
        if v:
            out[k] = np.frombuffer(v.to_bytes(4 * L, "little", signed=True), dtype="<u4")
    return out.reshape(nx, ny, L)


def _poly(arr):
    return _Poly(arr.shape[0] - 1, arr.shape[1] - 1, arr.shape[2],
                 arr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))


def _ints(rows_u32):
    """Signed integers from two's-complement rows [n][L] of uint32."""
    raw = np.ascontiguousarray(rows_u32, dtype="<u4")
    n, L = raw.shape
    b = raw.tobytes()
    return [int.from_bytes(b[4 * L * i:4 * L * (i + 1)], "little", signed=True) for i in range(n)]


def _check(rc, what):
    if rc:
        raise RuntimeError(f"O2 {what}: {O2_ERR.get(rc, rc)}")


def plan(f, g):
    """The oracle's plan of one pair: degrees, degree bound D, bits B, primes K."""
    lib = load()
    a, b = limbs_array(f), limbs_array(g)
    pl = _Plan()
    _check(lib.o2_plan_pair(ctypes.byref(_poly(a)), ctypes.byref(_poly(b)), ctypes.byref(pl)), "plan")
    return {n: getattr(pl, n) for n, _ in _Plan._fields_ if n != "pad"}


def prime(k):
    """The k-th prime of the oracle's own table (descending below 2^31 - 2^20)."""
    return int(load().o2_prime(k))


def resultants(pairs, threads=None, max_words=1 << 27, lib=None):
    """Res_y(f, g) of every pair as a list of Python ints (low to high, no
    trailing zeros; [] for zero), on ``threads`` host threads.  Pairs are
    taken in chunks whose residues stay under ``max_words`` 32-bit words."""
    lib = lib or load()
    threads = threads or os.cpu_count() or 1
    arrs = [(limbs_array(f), limbs_array(g)) for f, g in pairs]
    plans = []
    for a, b in arrs:
        pl = _Plan()
        _check(lib.o2_plan_pair(ctypes.byref(_poly(a)), ctypes.byref(_poly(b)), ctypes.byref(pl)), "plan")
        plans.append(pl)
    out = []
    i = 0
    while i < len(arrs):
        j, words = i, 0
        while j < len(arrs) and (j == i or words + plans[j].nprimes * (plans[j].D + 1) <= max_words):
            words += plans[j].nprimes * (plans[j].D + 1)
            j += 1
        out += _run(lib, arrs[i:j], plans[i:j], threads)
        i = j
    return out


def _run(lib, arrs, plans, threads):
    n = len(arrs)
    F = (_Poly * n)(*[_poly(a) for a, _ in arrs])
    G = (_Poly * n)(*[_poly(b) for _, b in arrs])
    bufs = [np.zeros(max(1, (pl.D + 1) * pl.out_limbs), dtype=np.uint32) for pl in plans]
    ptrs = (ctypes.POINTER(ctypes.c_uint32) * n)(*[b.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
                                                   for b in bufs])
    deg = (ctypes.c_int32 * n)()
    _check(lib.o2_resultant_batch(n, F, G, threads, ptrs, deg), "resultant")
    res = []
    for k, pl in enumerate(plans):
        d = deg[k]
        res.append([] if d < 0 else _ints(bufs[k][:(d + 1) * pl.out_limbs].reshape(d + 1, pl.out_limbs)))
    return res


def resultant(f, g, threads=None):
    return resultants([(f, g)], threads)[0]


def image(f, g, p, x, how=0):
    """det S(x) mod p by the batch's choice (how=0), the Sylvester matrix
    (1) or the Euclidean algorithm (2; raises where a leading coefficient
    vanishes at x)."""
    lib = load()
    a, b = limbs_array(f), limbs_array(g)
    rc = ctypes.c_int32()
    v = lib.o2_image(ctypes.byref(_poly(a)), ctypes.byref(_poly(b)), p, x % p, how, ctypes.byref(rc))
    _check(rc.value, "image")
    return int(v)


def residues(f, g, p):
    """R mod p (coefficients 0..D of the plan) from the images at x = 0..D."""
    lib = load()
    a, b = limbs_array(f), limbs_array(g)
    pl = plan(a, b)
    out = np.zeros(max(1, pl["D"] + 1), dtype=np.uint32)
    _check(lib.o2_residues(ctypes.byref(_poly(a)), ctypes.byref(_poly(b)), p,
                           out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))), "residues")
    return [int(v) for v in out]


def crt(res, bits):
    """Integers from residues res[k][c] modulo the first K table primes, in
    the symmetric range; every |value| must need at most bits + 1 bits."""
    lib = load()
    r = np.ascontiguousarray(res, dtype=np.uint32)
    K, n = r.shape
    Lo = (31 * K + 31) // 32
    out = np.zeros(max(1, n * Lo), dtype=np.uint32)
    _check(lib.o2_crt(K, n, r.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), bits, Lo,
                      out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))), "crt")
    return _ints(out[:n * Lo].reshape(n, Lo)) if n else []


def digest(R):
    """SHA-256 (hex) of the canonical text of a coefficient list: the degree,
    a semicolon, then every coefficient low to high in signed hexadecimal,
    comma-separated (no trailing zero coefficients)."""
    while R and R[-1] == 0:
        R = R[:-1]
    text = "%d;" % (len(R) - 1) + ",".join(format(c, "x") for c in R)
    return hashlib.sha256(text.encode()).hexdigest()
