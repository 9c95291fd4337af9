"""CPU-only checks of the C ABI: the library loads, exports every function
include/rs.h declares, and its host-side planner returns bounds that hold
for the oracle's exact results.  No GPU compute is called."""
import ctypes
import math
import os
import random
import re

import pytest

from oracle import exact
from paper_1010_1386_gb300 import inputs, rs
from tests.helpers import rand_bipoly

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "rs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rs_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(rs.LIB_PATH):
        from paper_1010_1386_gb300 import build
        build.build()
    return rs.load()


def test_exports_every_declared_function(lib):
    declared = header_functions()
    assert len(declared) >= 17
    for name in declared:
        assert hasattr(lib, name), name
    assert set(declared) == set(rs._SIGS), "binding and header disagree"


def test_error_strings(lib):
    assert lib.rs_error_string(0) == b"ok"
    assert lib.rs_error_string(-6).startswith(b"input exceeds")


def test_bounds_hold_for_oracle_results(lib):
    rng = random.Random(21)
    for _ in range(25):
        f = rand_bipoly(rng, rng.randint(0, 4), rng.randint(0, 4), bits=rng.choice([3, 30, 70]))
        g = rand_bipoly(rng, rng.randint(0, 4), rng.randint(0, 4), bits=rng.choice([3, 30, 70]))
        R = exact.resultant_y(f, g)
        b = rs.result_bound(f, g)
        assert len(R) - 1 <= b["deg"] <= exact.degree_bound(f, g)
        assert all(abs(c) < (1 << (b["bits"] - 1)) for c in R)
        assert b["limbs"] * 32 >= b["bits"]
        assert b["primes"] * 30.99 >= b["bits"] + 1


def test_bound_of_workloads(lib):
    [(f, g)] = inputs.workload_single(1)
    b = rs.result_bound(f, g)
    assert b["deg"] == 900 and 65 <= b["primes"] <= 80
    [(f, g)] = inputs.workload_small(0)
    assert rs.result_bound(f, g)["deg"] == 36


def _row_bound_exact(f):
    """H_f = a_0 + 2 sum_{k>=1} |a_k| with a_k = sum_j sum_i f_{j,i} f_{j,i+k}
    (f[i][j] the coefficient of x^i y^j) and the l1 form sum_j ||f_j||_1^2,
    in exact integers; the smaller of the two."""
    rows = [[f[i][j] for i in range(len(f))] for j in range(len(f[0]))]
    n = len(f)
    a = [sum(r[i] * r[i + k] for r in rows for i in range(n - k)) for k in range(n)]
    return min(a[0] + 2 * sum(abs(v) for v in a[1:]), sum(sum(abs(c) for c in r) ** 2 for r in rows))


def _bits_exact(f, g):
    """ceil(n_y/2 log2 H_f + m_y/2 log2 H_g) + 1, the planner's formula, by
    integer arithmetic: the smallest e with H_f^{n_y} H_g^{m_y} <= 4^(e - 1)."""
    my = max(j for r in f for j, c in enumerate(r) if c)
    ny = max(j for r in g for j, c in enumerate(r) if c)
    prod = _row_bound_exact(f) ** ny * _row_bound_exact(g) ** my
    e = 0
    while 4 ** e < prod:
        e += 1
    return e + 1


def test_row_norm_bound_matches_exact_integers(lib):
    """The planner's row bound (coefficients cut to 21 bits, floating sums
    with rounding margins) against the same formula in exact integers: the
    planner may only round up, by one bit at most, on single- and multi-limb
    coefficients, mixed magnitudes, sparse rows and all-positive rows (where
    the autocorrelation bound equals the l1 one)."""
    rng = random.Random(24)
    for case in range(120):
        kind = case % 4
        dx, dy = rng.randint(0, 12), rng.randint(1, 8)
        bits = rng.choice([4, 20, 31, 64, 100, 200])
        f = rand_bipoly(rng, dx, dy, bits=bits, density=0.3 if kind == 2 else 1.0)
        g = rand_bipoly(rng, rng.randint(0, 12), rng.randint(1, 8), bits=rng.choice([4, 40, 130]))
        if kind == 1:  # one huge coefficient among small ones
            f[rng.randint(0, dx)][rng.randint(0, dy)] = rng.choice([-1, 1]) << rng.randint(150, 300)
        if kind == 3:
            f = [[abs(c) for c in r] for r in f]
        b = rs.result_bound(f, g)
        want = _bits_exact(f, g)
        assert want <= b["bits"] <= want + 1, (case, want, b["bits"])
    # the widest coefficients the ABI takes (128 limbs), negative ones among them
    f = rand_bipoly(rng, 5, 3, bits=4000)
    g = rand_bipoly(rng, 4, 2, bits=2000)
    f[2][1] = -(1 << 4090) + 12345
    want = _bits_exact(f, g)
    assert want <= rs.result_bound(f, g)["bits"] <= want + 1


def test_row_norm_bound_holds_on_adversarial_pairs(lib):
    """Pairs whose resultants come close to the Hadamard-type bound (all
    coefficients positive, one dominant coefficient per row, y-degree one
    where R = f_1 g_0 - f_0 g_1) stay strictly inside it."""
    rng = random.Random(25)
    for case in range(40):
        dx = rng.randint(0, 6)
        if case % 3 == 0:
            f = [[rng.randint(1, 1 << 30) for _ in range(2)] for _ in range(dx + 1)]
            g = [[-rng.randint(1, 1 << 30), rng.randint(1, 1 << 30)] for _ in range(dx + 1)]
        elif case % 3 == 1:
            f = rand_bipoly(rng, dx, rng.randint(1, 4), bits=8)
            g = rand_bipoly(rng, dx, rng.randint(1, 4), bits=8)
            for p in (f, g):
                for j in range(len(p[0])):
                    p[rng.randint(0, dx)][j] = 1 << 40
        else:
            f = [[rng.randint(0, 1000) for _ in range(rng.randint(2, 4))] for _ in range(dx + 1)]
            g = [[rng.randint(0, 1000) for _ in range(len(f[0]))] for _ in range(dx + 1)]
            f[dx][-1] = f[dx][-1] or 1
            g[dx][-1] = g[dx][-1] or 1
        R = exact.resultant_y(f, g)
        b = rs.result_bound(f, g)
        assert all(abs(c) < (1 << (b["bits"] - 1)) for c in R), case


def test_factor_bound_holds_for_oracle_factorisations(lib):
    """The square-free path lifts H_i = lc(R) R_i / lc(R_i) with primes for
    coefficients below 2^(bits + D + ceil(log2(D + 1) / 2) + 1) (the
    Landau-Mignotte bound with the leading-coefficient ratio, from the
    planner's bits and D).  On resultants with planted repeated factors
    (f = y - x, so Res_y(f, g) is g(x) up to sign, with g built from a square
    and a cyclotomic-rich product; and Res_y(p q^2, (pq)_y) of small random
    p, q) every H_i of the oracle's exact factorisation satisfies
    ||H_i||_1 <= 2^(deg R_i) ||R||_2 and stays below that bound."""
    from oracle import squarefree as sq
    from oracle.exact import zx_mul
    from paper_1010_1386_gb300.inputs import _dy, _from_dict, _mul_dict, _to_dict
    rng = random.Random(26)

    def poly_pow(a, k):
        out = [1]
        for _ in range(k):
            out = zx_mul(out, a)
        return out

    cases = []
    for gy in ([-1] + [0] * 14 + [1],                                         # y^15 - 1
               zx_mul(poly_pow([1, 1], 3), poly_pow([-1, 0, 1], 2)),           # (y+1)^3 (y^2-1)^2
               zx_mul(poly_pow([2, -3, 1], 2), [-1] + [0] * 20 + [1]),         # (y^2-3y+2)^2 (y^21-1)
               zx_mul(poly_pow([rng.randint(-9, 9), rng.randint(-9, 9), 3], 2), [5, 0, 7, 1])):
        cases.append(([[0, 1], [-1, 0]], [list(gy)]))  # f = y - x, g = gy(y)
    for _ in range(4):
        p = [[rng.randint(-4, 4) for _ in range(3)] for _ in range(2)]
        q = [[rng.randint(-4, 4) for _ in range(2)] for _ in range(2)]
        p[1][2] = q[1][1] = 1
        pq = _mul_dict(_to_dict(p), _to_dict(q))
        cases.append((_from_dict(_mul_dict(pq, _to_dict(q))), _from_dict(_dy(pq))))
    checked = 0
    for f, g in cases:
        R = exact.resultant_y(f, g)
        if len(R) < 2:
            continue
        b = rs.result_bound(f, g)
        D = b["deg"]
        bitsH = b["bits"] + D + math.ceil(0.5 * math.log2(D + 1)) + 1
        norm2 = math.isqrt(sum(c * c for c in R)) + 1
        c, facs = sq.squarefree(R)
        for _, Ri in facs:
            H = [R[-1] * v // Ri[-1] for v in Ri]
            assert all(R[-1] * v % Ri[-1] == 0 for v in Ri)
            assert sum(abs(v) for v in H) <= (1 << (len(Ri) - 1)) * norm2
            assert max(abs(v) for v in H) < (1 << bitsH)
            checked += 1
    assert checked >= 10


def test_planner_errors(lib):
    with pytest.raises(rs.RsError) as e:
        rs.result_bound(rand_bipoly(random.Random(1), 1, 72), [[1, 1]])
    assert e.value.code == -6
    assert rs.result_bound([[0]], [[1, 1]])["deg"] == -1


def test_create_without_gpu_fails_cleanly(lib):
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        pytest.skip("a GPU is present")
    with pytest.raises(rs.RsError) as e:
        rs.Context()
    assert e.value.code == -4


def test_autotune_cache_file_roundtrip(lib, tmp_path):
    """The tuner cache is host state: a file merges into it, is written back
    in the same form, and a malformed line rejects the whole file."""
    rs.autotune_clear()
    assert rs.autotune_entries() == []
    good = tmp_path / "tune.txt"
    good.write_text("# comment\n"
                    "0 152 40 10 21 64 1 3.5 3.75\n"
                    "0 152 8 5 9 32 0 0.125 0.25\n"
                    "\n"
                    "0 148 72 13 24 128 1 0 0\n"
                    "1 152 0 12 22 1 0 2.5 3\n")
    rs.autotune_load(str(good))
    key = lambda e: (e["kind"], e["sms"], e["cap"], e["lg_points"], e["lg_images"])
    got = {key(e): e for e in rs.autotune_entries()}
    assert set(got) == {(0, 152, 40, 10, 21), (0, 152, 8, 5, 9), (0, 148, 72, 13, 24), (1, 152, 0, 12, 22)}
    e = got[(0, 152, 40, 10, 21)]
    assert (e["choice"], e["persistent"], e["ms_best"], e["ms_default"]) == (64, 1, 3.5, 3.75)
    assert (got[(0, 152, 8, 5, 9)]["choice"], got[(0, 152, 8, 5, 9)]["persistent"]) == (32, 0)
    assert got[(1, 152, 0, 12, 22)]["choice"] == 1
    out = tmp_path / "out.txt"
    rs.autotune_save(str(out))
    rs.autotune_clear()
    assert rs.autotune_entries() == []
    rs.autotune_load(str(out))
    again = {key(e): e for e in rs.autotune_entries()}
    assert again == got
    bad_lines = ["0 152 40 10 21 48 1 1 1",      # tile width not 32/64/128
                 "0 152 44 10 21 64 1 1 1",      # capacity not a multiple of 8
                 "0 152 40 10 21 64 2 1 1",      # schedule not 0/1
                 "1 152 0 12 22 3 0 1 1",        # G2 form not 0/1/2
                 "1 152 8 12 22 1 0 1 1",        # G2 entry with a capacity
                 "2 152 40 10 21 64 1 1 1",      # unknown kind
                 "0 152 40 10 21 64 1 1",        # a field missing
                 "0 152 40 10 21 64 1 1 1 9"]    # a field extra
    for i, line in enumerate(bad_lines):
        bad = tmp_path / f"bad{i}.txt"
        bad.write_text("0 152 16 6 10 128 1 1 1\n" + line + "\n")
        with pytest.raises(rs.RsError) as ei:
            rs.autotune_load(str(bad))
        assert ei.value.code == -1 and ":2:" in str(ei.value)
        assert len(rs.autotune_entries()) == 4, "a rejected file merges nothing"
    with pytest.raises(rs.RsError):
        rs.autotune_load(str(tmp_path / "missing.txt"))
    rs.autotune_clear()


def test_config_layout(lib):
    cfg = rs.rs_config()
    assert lib.rs_config_default(cfg) == 0
    assert (cfg.device, cfg.tile_points, cfg.use_graphs, cfg.persistent, cfg.timing, cfg.autotune) == \
        (-1, 0, 1, 1, 0, 1)
    assert cfg.mem_limit_bytes == 0 and cfg.autotune_cache is None
    assert cfg.g2_form == 0 and cfg.crt_form == 0
    assert rs.rs_config.mem_limit_bytes.offset == 32 and rs.rs_config.autotune_cache.offset == 40
    assert rs.rs_config.crt_form.offset == 48 and ctypes.sizeof(rs.rs_config) == 56


def test_info_struct_layouts(tmp_path):
    """The binding's ctypes structs match the header as a C compiler lays it
    out (sizes and field offsets)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    src = tmp_path / "layout.c"
    checks = [("rs_batch_info", rs.rs_batch_info), ("rs_sqf_info", rs.rs_sqf_info),
              ("rs_int_peak", rs.rs_int_peak)]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rs.h"', "int main(void) {"]
    for name, st in checks:
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for fname, _ in st._fields_:
            lines.append(f'  printf("{name}.{fname} %zu\\n", offsetof({name}, {fname}));')
    lines.append("  return 0;\n}")
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                  text=True).stdout.splitlines())
    for name, st in checks:
        assert int(got[name]) == ctypes.sizeof(st), name
        for fname, _ in st._fields_:
            assert int(got[f"{name}.{fname}"]) == getattr(st, fname).offset, (name, fname)
