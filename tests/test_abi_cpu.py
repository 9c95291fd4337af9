"""CPU-only checks of the C ABI: the library loads, exports every function
include/rs.h declares, and its host-side planner returns bounds that hold
for the oracle's exact results.  No GPU compute is called."""
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
    assert b["deg"] == 900 and 70 <= b["primes"] <= 80
    [(f, g)] = inputs.workload_small(0)
    assert rs.result_bound(f, g)["deg"] == 36


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
