"""H_eff psi at L=30 (the bench's orbital count and MPO) against the oracle.

The library builds its own environments on the GPU from the same seeded
integrals and MPS (D=256, mid-chain cut 14) that the oracle used for
golden/l30_slice.npz (written by golden/make_l30_slice.py from the oracle
only), and applies H_eff (Sec. II.B step 2) to the seeded two-site vector
kept on the three largest sectors.  Every output element is compared:
FP64 within 1e-12 of max|y|; BF16x3 within 1e-4 of the product of absolute
values; sliced within 2^-24 of the product of 64-block row maxima (the error
models of test_gpu_mixed.py and test_gpu_sliced.py).  Zero input outside
the slice must give zero output wherever no operator block reaches it.
"""
import os

import numpy as np
import pytest

import inputs
import paper_2412_04676_gb300 as g

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def case():
    from paper_2412_04676_gb300 import build
    build.build()
    gd = np.load(os.path.join(HERE, "golden", "l30_slice.npz"))
    L, N, tsz, D, b, s_int, s_mps, s_psi = (int(v) for v in gd["params"])
    h, eri = inputs.make_integrals(L, s_int)
    sites, dims = inputs.make_mps(L, N, tsz, D, s_mps, n_left=b)
    ctx = g.Context(L, N, tsz, D=D, autotune=False)
    ctx.load_integrals(h, eri)
    ctx.import_mps(sites, [0] * b + [1] * (L - b))
    ctx.build_envs(b)
    yield ctx, b, gd
    ctx.close()


def test_sector_table_matches_the_oracle(case):
    ctx, b, gd = case
    secs, info = ctx.tables(b)
    assert [[s["q"][0], s["q"][1], s["rows"], s["cols"]] for s in secs] == gd["sectors"].tolist()
    assert info["dim"] == gd["x"].size and info["n_terms"] > 1000


@pytest.mark.parametrize("form", ["fp64", "bf16x3", "sliced"])
def test_three_sector_slice_elementwise(case, form):
    ctx, b, gd = case
    x, y = gd["x"], gd["y"]
    prec = {"fp64": g.FP64, "bf16x3": g.MIXED_BF16X3, "sliced": g.SLICED_BF16}[form]
    out = ctx.apply_heff(b, x, precision=prec)
    err = np.abs(out - y)
    if form == "fp64":
        bound = 1e-12 * np.abs(y).max() + 0.0 * y
    elif form == "bf16x3":
        bound = 1e-4 * gd["abs_product"]
    else:
        bound = 2.0 ** -24 * gd["inflated_product"]
    assert np.all(err <= bound + 1e-300), (form, err.max(), (err / np.maximum(bound, 1e-300)).max())
    # outputs no operator block reaches stay exactly zero
    assert np.all(out[gd["abs_product"] == 0] == 0)
