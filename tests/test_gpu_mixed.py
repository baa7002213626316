"""Mixed-precision (BF16x3 split, FP32 accumulation, FP64 split-K reduction)
H_eff products on the tensor cores, against the FP64 path and the oracle.

Error model (stated bound): each operand is split x = hi + lo with
|x - hi - lo| <= 2^-18 |x|; a product keeps hi*hi + hi*lo + lo*hi, dropping
lo*lo <= 2^-18 |a b|; the phase-1 output X is re-split (2^-18) and its
FP32 sum runs over one block dimension in steps of 16 (at most 3 * 64
roundings of 2^-24 for blocks up to 1024).  Two-kernel form: the tensor
cores sum at most 8 chunks of 64 in FP32 before each promotion (<= 512 *
2^-24 per sum), the promotions of one split-K item add in FP32 (a few tens,
2^-24 each).  Fused kernel: one split-K item sums at most 32 chunks of 64
(K = 2048) in TMEM, 3 * 128 roundings of 2^-24.  Items add in FP64.
Elementwise |y_mixed - y| <= c * (|O^Lx| |psi| |O^xR|^T) with c = 1e-4
covers 3 * 2^-16 + 600 * 2^-24 with margin.
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


@pytest.mark.parametrize("fused", [True, False])
@pytest.mark.parametrize("L,N,tsz,D,seed,b", [
    (6, 6, 0, 16, 500, 2), (8, 7, 1, 40, 501, 3), (10, 10, 0, 200, 502, 4), (10, 9, 1, 150, 503, 7),
])
def test_mixed_product_within_bound(L, N, tsz, D, seed, b, fused):
    # autotune off: the tuner's trial products use different split-K
    # orders, and the last check below wants bitwise repeatability
    c = heff_case(L, N, tsz, D, seed, b, autotune=False, bf16x3_fused=fused)
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


@pytest.mark.parametrize("L,N,tsz,D,seed,b", [(10, 10, 0, 200, 502, 4), (12, 11, 1, 300, 504, 5)])
def test_fused_and_two_phase_products_agree(L, N, tsz, D, seed, b):
    # the fused kernel (X kept on the SM) and the two-kernel form compute the
    # same split products in different summation orders: both within the
    # stated accuracy of the FP64 product, and within twice of each other
    a = heff_case(L, N, tsz, D, seed, b, oracle=False, autotune=False, bf16x3_fused=True)
    t = heff_case(L, N, tsz, D, seed, b, oracle=False, autotune=False, bf16x3_fused=False)
    rng = np.random.default_rng(seed)
    x = rng.normal(size=a["ctx"].tables(b)[1]["dim"])
    y64 = a["ctx"].apply_heff(b, x, precision=g.FP64)
    yf = a["ctx"].apply_heff(b, x, precision=g.MIXED_BF16X3)
    yt = t["ctx"].apply_heff(b, x, precision=g.MIXED_BF16X3)
    yc = a["ctx"].apply_heff(b, x, precision=g.BF16X3_TWO_PHASE)  # comparison form on the fused context
    assert np.array_equal(yf, t["ctx"].apply_heff(b, x, precision=g.BF16X3_FUSED))  # and the other way round
    assert np.array_equal(y64, t["ctx"].apply_heff(b, x, precision=g.FP64))
    nrm = np.linalg.norm(y64)
    assert np.linalg.norm(yf - y64) <= 2e-5 * nrm
    assert np.linalg.norm(yt - y64) <= 2e-5 * nrm
    assert np.linalg.norm(yf - yt) <= 4e-5 * nrm
    assert np.array_equal(yc, yt)  # same kernels, same work list
    assert not np.array_equal(yf, yt)  # two different kernels really ran
    # back to the context's fused form after the comparison product
    assert np.array_equal(yf, a["ctx"].apply_heff(b, x, precision=g.MIXED_BF16X3))


def test_mixed_davidson_refines_below_the_bf16x3_floor():
    # BF16x3 products alone stall near 1e-5 |E| (~1e-4 here); after an anchor
    # the subspace holds the exact pair and its projections are taken on the
    # accurate side, so further mixed directions refine the exact residual:
    # the mixed Davidson reaches a tolerance far below the BF16x3 floor, with
    # the FP64 energy
    L, N, tsz, D, b = 10, 10, 0, 200, 4
    ref = heff_case(L, N, tsz, D, 530, b, oracle=False, dav_tol=1e-10)
    mix = heff_case(L, N, tsz, D, 530, b, oracle=False, dav_tol=1e-7, precision=g.MIXED_BF16X3)
    e64, _, _, rc64 = ref["ctx"].davidson(b)
    em, _, st, rc = mix["ctx"].davidson(b)
    assert rc64 == 0 and rc == 0, (rc, st["anchors"], st["anchor_resid"])
    assert st["resid"] <= 1e-7 and abs(em - e64) <= 1e-7, (em, e64, st)
    assert st["anchors"] >= 1
