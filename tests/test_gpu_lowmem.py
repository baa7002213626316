"""The mixed form's low-memory mode (gbd_config.low_memory = 1).

With sliced anchors the mixed Davidson reads only the tensor-core operator
planes, so the FP64 enlarged operators can be released once both forms'
planes exist (this is what lets the L=54, D=2048 workload fit the device).
Forced here at small sizes, the mode must not change any result: the
BF16x3 and sliced products are bitwise those of the normal mode, an FP64
product afterwards enlarges the operators again and matches the oracle
(Sec. II.B step 2), the renormalisation runs on the sliced planes alone
(Sec. II.B step 3), and whole steps give the same energies.
"""
import numpy as np
import pytest

import inputs
import paper_2412_04676_gb300 as g
from gpu_common import build_lib, heff_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    build_lib()


def test_low_memory_products_are_unchanged():
    L, N, tsz, D, b = 10, 10, 0, 150, 4
    out = {}
    for lm in (-1, 1):
        c = heff_case(L, N, tsz, D, 610, b, oracle=(lm == 1), precision=g.MIXED_BF16X3, low_memory=lm,
                      autotune=False)
        ctx = c["ctx"]
        secs, info = ctx.tables(b)
        x = np.random.default_rng(1).normal(size=info["dim"])
        ym = ctx.apply_heff(b, x, precision=g.MIXED_BF16X3)
        ys = ctx.apply_heff(b, x, precision=g.SLICED_BF16)
        y64 = ctx.apply_heff(b, x, precision=g.FP64)   # low-memory: enlarges again
        ym2 = ctx.apply_heff(b, x, precision=g.MIXED_BF16X3)
        out[lm] = (ym, ys, y64, ym2, c["He"])
        ctx.close()
    for k in range(3):
        assert np.array_equal(out[-1][k], out[1][k])
    assert np.array_equal(out[1][0], out[1][3])
    # the mixed form enlarges with sliced tensor-core GEMMs (about 2^-30 of
    # the block maxima), so its FP64 product matches the oracle to ~1e-9
    He = out[1][4]
    y_ref = He.matvec(np.random.default_rng(1).normal(size=He.dim))
    assert np.abs(out[1][2] - y_ref).max() <= 1e-8 * np.abs(y_ref).max()


def test_low_memory_steps_give_the_same_energies():
    L, N, tsz, D, b = 10, 10, 0, 120, 4
    h, eri = inputs.make_integrals(L, 620)
    sites, dims = inputs.make_mps(L, N, tsz, D, 621, n_left=b)
    res = {}
    for lm in (-1, 1):
        c = g.Context(L, N, tsz, D=D, precision=g.MIXED_BF16X3, low_memory=lm, offload=True, dav_tol=1e-7,
                      autotune=False)
        c.load_integrals(h, eri)
        c.import_mps(sites, [0] * b + [1] * (L - b))
        c.build_envs(b)
        es = []
        for (p, d) in ((b, 1), (b + 1, 1), (b + 2, -1), (b + 1, -1)):
            es.append(c.step(p, d, D)["energy"])
        res[lm] = (np.array(es), c.env_export(0, b + 1))
        c.close()
    assert np.abs(res[1][0] - res[-1][0]).max() <= 1e-12
    assert np.array_equal(res[1][1], res[-1][1])
