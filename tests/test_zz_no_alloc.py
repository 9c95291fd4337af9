"""rs_crt_noalloc: the CRT entry point that allocates nothing, for callers
that may not allocate device memory themselves or through the library (a
plugin handed fixed buffers, code where cudaMalloc/cudaFree could
synchronise the device or fail).  Its output must equal the regular
resultant path's, bit for bit, on two calls in a row that share its fixed
scratch array, and equal the oracle's.  The test itself allocates the input
and output buffers with torch, as such a caller's host application would."""
import ctypes
import random

import numpy as np
import pytest

from paper_1010_1386_gb300 import rs
from oracle import exact
from tests.helpers import rand_bipoly

pytestmark = pytest.mark.gpu


def _residues(R, primes, N):
    res = np.zeros((len(primes), N), dtype=np.uint32)
    for k, p in enumerate(primes):
        for j, c in enumerate(R):
            res[k, j] = c % p
    return res


def _run_noalloc(lib, torch, res, L):
    K, N = res.shape
    d_res = torch.from_numpy(res.view(np.int32).copy()).cuda()
    d_out = torch.zeros(N * L, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.rs_crt_noalloc(ctypes.c_void_p(d_res.data_ptr()), K, N, L,
                            ctypes.c_void_p(d_out.data_ptr()), ctypes.c_void_p(stream))
    assert rc == 0
    torch.cuda.synchronize()
    out = d_out.cpu().numpy().view(np.uint32).reshape(N, L)
    return [int.from_bytes(row.astype("<u4").tobytes(), "little", signed=True) for row in out]


def test_noalloc_crt_matches_resultant_path_and_oracle():
    """Two calls in a row (different sizes, one shared scratch array): the
    residues of the oracle's R modulo the library's primes come back as R,
    equal to the regular resultant path's output."""
    torch = pytest.importorskip("torch")
    lib = rs.load()
    ctx = rs.Context(device=0)
    rng = random.Random(31)
    cases = [(rand_bipoly(rng, 4, 5, bits=40), rand_bipoly(rng, 3, 6, bits=40)),
             (rand_bipoly(rng, 6, 3, bits=100), rand_bipoly(rng, 5, 4, bits=100))]
    for f, g in cases:
        R = exact.resultant_y(f, g)
        b = rs.result_bound(f, g)
        K, N, L = b["primes"], b["deg"] + 1, b["limbs"]
        primes, _, _ = ctx.images(f, g, K, 1)
        got = _run_noalloc(lib, torch, _residues(R, [int(p) for p in primes], N), L)
        assert got == list(R) + [0] * (N - len(R))
        assert ctx.resultant_y(f, g) == R
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = rs.load()
    # both are refused on the host before any device work
    assert lib.rs_crt_noalloc(ctypes.c_void_p(256), 4096, 10, 1, ctypes.c_void_p(256), None) == -6
    assert lib.rs_crt_noalloc(ctypes.c_void_p(256), 100, 30000, 100, ctypes.c_void_p(256), None) == -6
    assert lib.rs_crt_noalloc(None, 1, 1, 1, None, None) == -1


def test_noalloc_crt_random_residues_vs_python():
    """The CRT kernels on arbitrary residues (not images of a resultant):
    the output is the unique integer in the symmetric range (-P/2, P/2)
    congruent to every residue, P the product of the first K table primes;
    residues 0, p - 1 and (p +- 1)/2 included, K from 1 to 1000."""
    torch = pytest.importorskip("torch")
    lib = rs.load()
    ctx = rs.Context(device=0)
    rng = random.Random(32)
    table, _, _ = ctx.images([[0, 1]], [[1, 1], [1]], 1000, 1)
    table = [int(p) for p in table]
    for K, N in [(1, 5), (2, 9), (7, 33), (64, 40), (65, 17), (200, 64), (1000, 6)]:
        primes = table[:K]
        P = 1
        for p in primes:
            P *= p
        L = (P.bit_length() + 1 + 31) // 32
        res = np.zeros((K, N), dtype=np.uint32)
        for j in range(N):
            for k, p in enumerate(primes):
                res[k, j] = rng.choice([0, p - 1, (p - 1) // 2, (p + 1) // 2, rng.randrange(p)])
        got = _run_noalloc(lib, torch, res, L)
        for j in range(N):
            x = 0
            for k, p in enumerate(primes):  # Garner-free CRT by the explicit formula
                Pk = P // p
                x = (x + int(res[k, j]) * Pk * pow(Pk, -1, p)) % P
            if x > P // 2:
                x -= P
            assert got[j] == x, (K, j)
    ctx.close()


def test_noalloc_at_the_scratch_limit_and_the_prime_limit():
    """nprimes * ncoeffs + ncoeffs * limbs exactly 2^21 (the last limb lands
    on the scratch array's last word), then nprimes = 2048, the largest
    table prefix: known integers in the symmetric range come back exactly."""
    torch = pytest.importorskip("torch")
    lib = rs.load()
    ctx = rs.Context(device=0)
    rng = random.Random(33)
    table, _, _ = ctx.images([[0, 1]], [[1, 1], [1]], 2048, 1)
    table = [int(p) for p in table]
    for K, N, L in [(1000, 1024, 1048), (2048, 8, 1990)]:
        assert K * N + N * L <= 1 << 21
        P = 1
        for p in table[:K]:
            P *= p
        vals = [rng.randrange(-(P // 2), P // 2 + 1) for _ in range(13)] + [0, 1, -1, P // 2, -(P // 2)]
        pick = [vals[(7 * j + 3) % len(vals)] for j in range(N)]
        rows = {v: [v % p for p in table[:K]] for v in vals}
        res = np.zeros((K, N), dtype=np.uint32)
        for j, v in enumerate(pick):
            res[:, j] = rows[v]
        got = _run_noalloc(lib, torch, res, L)
        assert got == pick, K
    assert 1000 * 1024 + 1024 * 1048 == 1 << 21
    ctx.close()
