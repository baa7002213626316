"""Mixed-precision (BF16x3 split, FP32 accumulation, FP64 split-K reduction)
H_eff products on the tensor cores, against the FP64 path and the oracle.

Error model (stated bound): each operand is split x = hi + lo with
|x - hi - lo| <= 2^-18 |x|; a product keeps hi*hi + hi*lo + lo*hi, dropping
lo*lo <= 2^-18 |a b|; the phase-1 output is re-split (2^-18); the tensor
cores sum at most 8 chunks of 64 in FP32 before each promotion (<= 512 *
2^-24 per sum), the promotions of one split-K item add in FP32 (a few tens,
2^-24 each) and the items in FP64.  Elementwise
|y_mixed - y| <= c * (|O^Lx| |psi| |O^xR|^T) with c = 1e-4 covers
3 * 2^-16 + 600 * 2^-24 with margin.
"""
import numpy as np
import pytest

import inputs
import paper_2412_04676_gb300 as g
from gpu_common import build_lib, heff_case
from oracle import dmrg as R
from oracle import hamiltonian as H
from oracle import mpo as M

pytestmark = pytest.mark.gpu
C_BOUND = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    build_lib()


def _abs_product(He, x):
    """|O^Lx| |psi| |O^xR|^T with the oracle's operators (elementwise bound)."""
    psi = He.unflatten(np.abs(x))
    Y = {Q: np.zeros(s) for Q, s in He.shape.items()}
    for (Q, Q2), bl, br in He.pairs:
        X = np.einsum("cij,jk->cik", np.abs(bl), psi[Q2])
        Y[Q] += np.einsum("cik,clk->il", X, np.abs(br))
    return He.flatten(Y)


@pytest.mark.parametrize("L,N,tsz,D,seed,b", [
    (6, 6, 0, 16, 500, 2), (8, 7, 1, 40, 501, 3), (10, 10, 0, 200, 502, 4), (10, 9, 1, 150, 503, 7),
])
def test_mixed_product_within_bound(L, N, tsz, D, seed, b):
    # autotune off: the tuner's trial products use different split-K
    # orders, and the last check below wants bitwise repeatability
    c = heff_case(L, N, tsz, D, seed, b, autotune=False)
    ctx, He = c["ctx"], c["He"]
    x = He.flatten(He.to_enlarged(c["psi4"], None))
    y64 = ctx.apply_heff(b, x, precision=g.FP64)
    ym = ctx.apply_heff(b, x, precision=g.MIXED_BF16X3)
    bound = C_BOUND * _abs_product(He, x)
    err = np.abs(ym - y64)
    assert np.all(err <= bound + 1e-300), (err.max(), (err / np.maximum(bound, 1e-300)).max())
    y_ref = He.matvec(x)
    assert np.abs(y64 - y_ref).max() <= 1e-12 * np.abs(y_ref).max()
    # repeated products are bitwise deterministic
    assert np.array_equal(ym, ctx.apply_heff(b, x, precision=g.MIXED_BF16X3))


@pytest.mark.parametrize("polish", [0, 1, 2])
def test_mixed_davidson_energy_within_1e6(polish):
    # anchors: none (then the bound is the mixed products' own accuracy),
    # FP64 products, sliced tensor-core products
    L, N, tsz, D, b = 10, 10, 0, 120, 4
    ref = heff_case(L, N, tsz, D, 510, b, dav_tol=1e-9)
    mix = heff_case(L, N, tsz, D, 510, b, oracle=False, dav_tol=1e-7, precision=g.MIXED_BF16X3,
                    mixed_polish=polish)
    x0 = ref["He"].flatten(ref["He"].to_enlarged(ref["psi4"], None))
    e64, _, _, _ = ref["ctx"].davidson(b, x0.copy())
    em, _, st, _ = mix["ctx"].davidson(b, x0.copy())
    assert abs(em - e64) <= (1e-3 if polish == 0 else 1e-6), (em, e64)


@pytest.mark.parametrize("polish", [1, 2])
def test_mixed_sweep_energy_within_1e6(polish):
    L, N, tsz, D = 10, 10, 0, 48
    h, eri = inputs.make_integrals(L, 520)
    sites, dims = inputs.make_mps(L, N, tsz, D, 521)
    out = {}
    for prec in (g.FP64, g.MIXED_BF16X3):
        ctx = g.Context(L, N, tsz, D=D, dav_tol=1e-7, precision=prec, mixed_polish=polish)
        ctx.load_integrals(h, eri)
        ctx.import_mps(sites, [1] * L)
        out[prec] = ctx.sweep(2, D)[-1]["energy_last"]
    assert abs(out[g.MIXED_BF16X3] - out[g.FP64]) <= 1e-6, out


def test_mixed_product_full_size_l30_d1024():
    # L=30, N=30, D=1024 at the mid-chain cut (the bench's launch configuration):
    # mixed vs the FP64 product of the same library, relative norm error and
    # the symmetry of the mixed operator (properties that hold at any size)
    L, N, tsz, D, b = 30, 30, 0, 1024, 14
    c = heff_case(L, N, tsz, D, 1002, b, oracle=False)
    ctx = c["ctx"]
    secs, info = ctx.tables(b)
    rng = np.random.default_rng(5)
    x = rng.normal(size=info["dim"])
    z = rng.normal(size=info["dim"])
    y64 = ctx.apply_heff(b, x, precision=g.FP64)
    ym = ctx.apply_heff(b, x, precision=g.MIXED_BF16X3)
    assert np.linalg.norm(ym - y64) <= 2e-5 * np.linalg.norm(y64)
    zm = ctx.apply_heff(b, z, precision=g.MIXED_BF16X3)
    assert abs(z @ ym - x @ zm) <= 2e-5 * np.linalg.norm(ym) * np.linalg.norm(z)
