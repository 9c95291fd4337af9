"""The G1 tuner (tile width and schedule per workload class) changes no
result: every candidate it can pick, and the tuned choice, give the oracle's
resultants; the cache it fills survives a round trip through its file."""
import os
import random

import numpy as np
import pytest

from oracle import exact
from paper_1010_1386_gb300 import rs
from tests.helpers import rand_bipoly

pytestmark = pytest.mark.gpu


def mixed_pairs(seed=11, n=40):
    """y-degrees spread over several register capacities (8, 16, 24) and
    point counts that leave ragged tiles of every width."""
    rng = random.Random(seed)
    pairs = []
    for _ in range(n):
        dy = rng.choice([1, 3, 7, 9, 12, 17, 20])
        dx = rng.randint(0, 4)
        bits = rng.choice([6, 30, 70])
        pairs.append((rand_bipoly(rng, dx, dy, bits=bits),
                      rand_bipoly(rng, rng.randint(0, 4), rng.randint(1, dy), bits=bits)))
    return pairs


def as_arrays(raw):
    return [(d, l, np.asarray(b[: (d + 1) * l]).copy()) for d, l, b in raw]


def same(a, b):
    return len(a) == len(b) and all(x[0] == y[0] and x[1] == y[1] and np.array_equal(x[2], y[2])
                                    for x, y in zip(a, b))


def test_every_candidate_gives_the_oracle_result():
    pairs = mixed_pairs()
    want = [exact.resultant_y(f, g) for f, g in pairs[:12]]
    base = None
    for width in (32, 64, 128):
        for persistent in (True, False):
            with rs.Context(device=0, tile_points=width, persistent=persistent) as ctx:
                got = as_arrays(ctx.resultant_batch(pairs, raw=True))
            ints = [rs.limbs_to_ints(b, d, l) for d, l, b in got[:12]]
            assert ints == want, (width, persistent)
            if base is None:
                base = got
            assert same(got, base), (width, persistent)


def test_tuned_batch_matches_and_fills_the_cache(tmp_path):
    pairs = mixed_pairs(seed=12)
    rs.autotune_clear()
    path = str(tmp_path / "tune.txt")
    with rs.Context(device=0, autotune_cache=path) as ctx:
        got = as_arrays(ctx.resultant_batch(pairs, raw=True))
        ent = rs.autotune_entries()
    caps = {e["cap"] for e in ent if e["kind"] == 0}
    assert {8, 16, 24} <= caps, ent
    for e in ent:
        if e["kind"] == 0:
            assert e["choice"] in (32, 64, 128) and e["persistent"] in (0, 1)
        else:
            assert e["choice"] in (0, 1) and e["persistent"] == 0
        assert e["ms_best"] > 0 and e["ms_default"] > 0
        assert e["ms_best"] <= e["ms_default"]
    assert os.path.exists(path), "the cache file is written when the context is destroyed"
    with rs.Context(device=0, autotune=False, tile_points=128) as ctx:
        ref = as_arrays(ctx.resultant_batch(pairs, raw=True))
    assert same(got, ref)
    for (f, g), (d, l, b) in zip(pairs[:8], got[:8]):
        assert rs.limbs_to_ints(b, d, l) == exact.resultant_y(f, g)

    # A new context reads the file back: the same choices, no re-timing.
    rs.autotune_clear()
    with rs.Context(device=0, autotune_cache=path) as ctx:
        assert sorted(map(lambda e: tuple(e.values()), rs.autotune_entries())) == \
            sorted(map(lambda e: tuple(e.values()), ent))
        again = as_arrays(ctx.resultant_batch(pairs, raw=True))
        assert sorted(map(lambda e: tuple(e.values()), rs.autotune_entries())) == \
            sorted(map(lambda e: tuple(e.values()), ent))
    assert same(again, got)


def test_explicit_autotune_then_server_uses_cache():
    pairs = mixed_pairs(seed=13, n=24)
    rs.autotune_clear()
    with rs.Context(device=0) as ctx:
        ctx.autotune(pairs)
        n = len(rs.autotune_entries())
        assert n >= 1
        srv = rs.Server(ctx)
        tickets = [srv.submit(f, g) for f, g in pairs]
        res = [srv.wait(t, timeout_us=60_000_000)[0] for t in tickets]
        srv.stop()
        assert len(rs.autotune_entries()) == n, "the server never tunes"
    for (f, g), r in zip(pairs[:8], res[:8]):
        assert r == exact.resultant_y(f, g)
