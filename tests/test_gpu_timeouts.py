"""Failure detection of the tensor-core kernels without a GPU fault.

Every mbarrier wait in the tcgen05 kernels (G2 products, CRT digits) gives up
after about a second, drains the block's copies and MMAs, frees its tensor
memory and sets the batch's status word, which the host turns into
RS_ERR_TIMEOUT.  The test hook rs_test_stall_tensor_cores makes the copy
warps issue nothing (a flag that nothing else sets), so the waits run out;
the context must then report the timeout promptly and, with the hook off,
give exact results again.  No kernel faults, traps or hangs.
"""
import random
import time

import pytest

from oracle import exact
from paper_1010_1386_gb300 import rs
from tests.helpers import rand_bipoly

pytestmark = pytest.mark.gpu

RS_ERR_TIMEOUT = -5


def _expect_timeout_then_recover(ctx, pairs):
    want = [exact.resultant_y(f, g) for f, g in pairs]
    assert ctx.resultant_batch(pairs) == want  # the shapes run normally first
    ctx.stall_tensor_cores(True)
    t0 = time.time()
    with pytest.raises(rs.RsError) as ei:
        ctx.resultant_batch(pairs)
    assert ei.value.code == RS_ERR_TIMEOUT
    assert time.time() - t0 < 60
    ctx.stall_tensor_cores(False)
    assert ctx.resultant_batch(pairs) == want


def test_g2_products_wait_runs_out_and_context_recovers():
    rng = random.Random(61)
    pairs = [(rand_bipoly(rng, 2, 3, bits=20), rand_bipoly(rng, 2, 3, bits=20)) for _ in range(3)]
    with rs.Context(device=0, g2_form=4) as c:
        _expect_timeout_then_recover(c, pairs)


def test_crt_digit_wait_runs_out_and_context_recovers():
    rng = random.Random(62)
    pairs = [(rand_bipoly(rng, 1, 2, bits=700), rand_bipoly(rng, 1, 2, bits=700))]
    assert rs.result_bound(*pairs[0])["primes"] > 64  # two digit blocks: the copy warp has work
    with rs.Context(device=0, crt_form=2) as c:
        _expect_timeout_then_recover(c, pairs)
