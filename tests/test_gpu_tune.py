"""The autotuner of the BF16x3 H_eff product (tile shapes picked over the
measured sector-size distribution).

At a new position the first BF16x3 products try the candidate phase-2 work
list shapes (split-K items per SM, item order) one after another, each timed
on the device; the fastest is kept and cached under a key made from the
sector-size histogram.  Every candidate computes the same product (only the
FP32 partial sums are grouped differently, each reduced in FP64), so all
products agree far inside the BF16x3 error; a second context at a position
with the same histogram takes the cached choice without trials.
"""
import numpy as np
import pytest

import paper_2412_04676_gb300 as g
from gpu_common import build_lib, heff_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    build_lib()


def test_tuner_tries_every_candidate_then_keeps_the_fastest():
    # the tuner's cache is shared by every context of the process: start empty
    g.tune_reset()
    L, N, tsz, D, b = 10, 10, 0, 190, 4
    c = heff_case(L, N, tsz, D, 700, b, oracle=False)
    ctx = c["ctx"]
    secs, info = ctx.tables(b)
    x = np.random.default_rng(2).normal(size=info["dim"])
    y64 = ctx.apply_heff(b, x, precision=g.FP64)
    ys = []
    ti = None
    for i in range(8):
        ys.append(ctx.apply_heff(b, x, precision=g.MIXED_BF16X3))
        ti = ctx.tune_info()
        if i < len(ti["candidates"]) - 1:
            assert ti["active"] and ti["current"] == i + 1
    n = len(ti["candidates"])
    assert not ti["active"] and 0 <= ti["chosen"] < n and not ti["from_cache"]
    ms = [cd["ms"] for cd in ti["candidates"]]
    assert all(m > 0 for m in ms) and ti["chosen"] == int(np.argmin(ms))
    assert sum(ti["hist"]) == len(secs)
    scale = np.abs(y64).max()
    for y in ys:
        assert np.abs(y - ys[0]).max() <= 1e-9 * scale      # same product, other grouping
        assert np.linalg.norm(y - y64) <= 2e-5 * np.linalg.norm(y64)
    # the chosen shape stays: later products are bitwise repeatable
    assert np.array_equal(ys[-1], ys[-2])
    ctx.close()
    # same position, fresh context: the cached choice, no trials
    c2 = heff_case(L, N, tsz, D, 700, b, oracle=False)
    ctx2 = c2["ctx"]
    ctx2.tables(b)
    ctx2.apply_heff(b, x, precision=g.MIXED_BF16X3)
    t2 = ctx2.tune_info()
    assert t2["from_cache"] and not t2["active"] and t2["chosen"] == ti["chosen"] and t2["key"] == ti["key"]
    ctx2.close()


def test_autotune_off_uses_the_fixed_shape():
    L, N, tsz, D, b = 8, 8, 0, 60, 3
    c = heff_case(L, N, tsz, D, 701, b, oracle=False, autotune=False)
    ctx = c["ctx"]
    secs, info = ctx.tables(b)
    ctx.apply_heff(b, np.ones(info["dim"]), precision=g.MIXED_BF16X3)
    t = ctx.tune_info()
    assert t["current"] == -1 and t["chosen"] == -1 and not t["active"]
    ctx.close()
