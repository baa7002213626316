"""Sliced (error-free splitting, ten BF16 products) H_eff products on the
tensor cores, against the FP64 path and the oracle.

Error model (stated bound).  Every operand row is cut into 64-wide K blocks;
a block whose maximum magnitude is below 2^e is written as four BF16 slices
on the grids 2^(e-8), ..., 2^(e-32), so the dropped remainder is at most
2^-32 of the block maximum.  The products keep slice pairs of order <= 4; the
dropped orders are below 2^-32 of (row block max) x (column block max) per
term.  Orders 1 and 2 accumulate exactly in FP32 inside a block; the rounded
add of orders 3-4 costs 2^-24 of a 2^-8 quantity.  The phase-1 output is
re-sliced per 64-column block (2^-32 of the block maximum).  So with every
matrix replaced by its 64-block row maxima ("inflated"), elementwise
|y_sliced - y| <= c * sum_t inflate(|O^L_t|inf |psi|inf) |O^R_t|inf^T, where
c = 2^-24 leaves a factor 256 over the ~2^-32 per-term error for the number
of error terms and for the library's operator sets differing from the
oracle's.  The BF16x3 form (2^-16 relative) fails this bound by orders of
magnitude.
"""
import numpy as np
import pytest

import inputs
import paper_2412_04676_gb300 as g
from gpu_common import build_lib, heff_case

pytestmark = pytest.mark.gpu
C_BOUND = 2.0 ** -24


@pytest.fixture(scope="module", autouse=True)
def built():
    build_lib()


def _inflate(a, axis):
    """Replace every entry by the maximum |entry| of its 64-block along axis."""
    a = np.moveaxis(np.abs(a), axis, -1)
    n = a.shape[-1]
    nb = -(-n // 64)
    pad = np.zeros(a.shape[:-1] + (nb * 64 - n,))
    m = np.concatenate([a, pad], axis=-1).reshape(a.shape[:-1] + (nb, 64)).max(axis=-1)
    out = np.repeat(m, 64, axis=-1)[..., :n]
    return np.moveaxis(out, -1, axis)


def _inflated_product(He, x):
    psi = He.unflatten(x)
    Y = {Q: np.zeros(s) for Q, s in He.shape.items()}
    for (Q, Q2), bl, br in He.pairs:
        X = np.einsum("cij,jk->cik", _inflate(bl, 2), _inflate(psi[Q2], 0))
        Y[Q] += np.einsum("cik,clk->il", _inflate(X, 2), _inflate(br, 2))
    return He.flatten(Y)


@pytest.mark.parametrize("L,N,tsz,D,seed,b", [
    (6, 6, 0, 16, 500, 2), (8, 7, 1, 40, 501, 3), (10, 10, 0, 200, 502, 4), (10, 9, 1, 150, 503, 7),
])
def test_sliced_product_within_bound(L, N, tsz, D, seed, b):
    c = heff_case(L, N, tsz, D, seed, b)
    ctx, He = c["ctx"], c["He"]
    x = He.flatten(He.to_enlarged(c["psi4"], None))
    y_ref = He.matvec(x)
    ys = ctx.apply_heff(b, x, precision=g.SLICED_BF16)
    bound = C_BOUND * _inflated_product(He, x)
    err = np.abs(ys - y_ref)
    assert np.all(err <= bound + 1e-300), (err.max(), (err / np.maximum(bound, 1e-300)).max())
    # far tighter than the BF16x3 form
    ym = ctx.apply_heff(b, x, precision=g.MIXED_BF16X3)
    assert np.linalg.norm(ys - y_ref) <= 1e-3 * np.linalg.norm(ym - y_ref) + 1e-300
    # repeated products are bitwise deterministic
    assert np.array_equal(ys, ctx.apply_heff(b, x, precision=g.SLICED_BF16))


def test_sliced_edge_cases():
    # a zero vector gives an exact zero; a vector with one nonzero sector
    # gives the oracle's product of that sector within the bound
    L, N, tsz, D, b = 8, 8, 0, 60, 3
    c = heff_case(L, N, tsz, D, 530, b)
    ctx, He = c["ctx"], c["He"]
    secs, info = ctx.tables(b)
    z = np.zeros(info["dim"])
    assert np.array_equal(ctx.apply_heff(b, z, precision=g.SLICED_BF16), z)
    x = np.zeros(info["dim"])
    s = max(secs, key=lambda s: s["rows"] * s["cols"])
    rng = np.random.default_rng(3)
    # values spanning 30 binades inside one sector: the grid follows each block's maximum
    x[s["offset"]:s["offset"] + s["rows"] * s["cols"]] = rng.normal(size=s["rows"] * s["cols"]) * \
        np.exp2(rng.integers(-30, 1, size=s["rows"] * s["cols"]))
    y_ref = He.matvec(x)
    ys = ctx.apply_heff(b, x, precision=g.SLICED_BF16)
    bound = C_BOUND * _inflated_product(He, x)
    assert np.all(np.abs(ys - y_ref) <= bound + 1e-300)


def test_sliced_anchor_davidson_energy():
    # mixed Davidson whose anchors are sliced products: the energy matches
    # the FP64 Davidson far inside 1e-6
    L, N, tsz, D, b = 10, 10, 0, 120, 4
    ref = heff_case(L, N, tsz, D, 510, b, dav_tol=1e-9)
    mix = heff_case(L, N, tsz, D, 510, b, oracle=False, dav_tol=1e-7, precision=g.MIXED_BF16X3, mixed_polish=2)
    x0 = ref["He"].flatten(ref["He"].to_enlarged(ref["psi4"], None))
    e64, _, _, _ = ref["ctx"].davidson(b, x0.copy())
    es, _, st, _ = mix["ctx"].davidson(b, x0.copy())
    assert abs(es - e64) <= 1e-8, (es, e64, st)


def test_sliced_anchor_sweep_energy():
    L, N, tsz, D = 10, 10, 0, 48
    h, eri = inputs.make_integrals(L, 520)
    sites, dims = inputs.make_mps(L, N, tsz, D, 521)
    out = {}
    for prec, pol in ((g.FP64, 1), (g.MIXED_BF16X3, 2)):
        ctx = g.Context(L, N, tsz, D=D, dav_tol=1e-7, precision=prec, mixed_polish=pol)
        ctx.load_integrals(h, eri)
        ctx.import_mps(sites, [1] * L)
        out[prec] = ctx.sweep(2, D)[-1]["energy_last"]
    assert abs(out[g.MIXED_BF16X3] - out[g.FP64]) <= 1e-7, out


def test_sliced_product_full_size_l30_d1024():
    # L=30, N=30, D=1024 at the mid-chain cut (the bench's launch configuration):
    # sliced vs the FP64 product of the same library, relative norm error and
    # the symmetry of the sliced operator (properties that hold at any size)
    L, N, tsz, D, b = 30, 30, 0, 1024, 14
    c = heff_case(L, N, tsz, D, 1002, b, oracle=False)
    ctx = c["ctx"]
    secs, info = ctx.tables(b)
    rng = np.random.default_rng(5)
    x = rng.normal(size=info["dim"])
    z = rng.normal(size=info["dim"])
    y64 = ctx.apply_heff(b, x, precision=g.FP64)
    ys = ctx.apply_heff(b, x, precision=g.SLICED_BF16)
    assert np.linalg.norm(ys - y64) <= 1e-8 * np.linalg.norm(y64)
    zs = ctx.apply_heff(b, z, precision=g.SLICED_BF16)
    assert abs(z @ ys - x @ zs) <= 1e-8 * np.linalg.norm(ys) * np.linalg.norm(z)


@pytest.mark.parametrize("direction", [1, -1])
def test_sliced_renormalisation_matches_fp64(direction):
    # the same two-site vector truncated in two contexts: FP64 renormalisation
    # (mixed_polish=1) and phase A of it on the tensor cores in the sliced form
    # (mixed_polish=2); the eigensolve is FP64 in both, so the kept bases agree
    # and the renormalised environments differ by the sliced rounding only
    L, N, tsz, D, b = 10, 10, 0, 80, 4
    out = {}
    for polish in (1, 2):
        c = heff_case(L, N, tsz, D, 540, b, oracle=False, precision=g.MIXED_BF16X3, mixed_polish=polish)
        ctx = c["ctx"]
        secs, info = ctx.tables(b)
        x = np.random.default_rng(7).normal(size=info["dim"])
        x /= np.linalg.norm(x)
        ctx.apply_heff(b, x, precision=g.SLICED_BF16)  # builds this position's sliced planes
        ctx.set_psi(b, x)
        ctx.truncate(b, direction, 40)
        tm = ctx.timers()
        assert (tm["renorm_tc_gflop"] > 0) == (polish == 2), tm  # the tensor-core path ran exactly when asked
        out[polish] = ctx.env_export(0 if direction == 1 else 1, b + 1)
    assert out[1].shape == out[2].shape and out[1].size > 0
    assert np.linalg.norm(out[2] - out[1]) <= 1e-8 * np.linalg.norm(out[1])


def test_sliced_enlargement_matches_fp64():
    # the environments and enlarged blocks of one position built in two
    # contexts: FP64 coefficient GEMMs (mixed_polish=1) and the same GEMMs on
    # the tensor cores in the sliced form (mixed_polish=2).  The FP64 H_eff
    # product then differs only through the enlargement's sliced rounding.
    L, N, tsz, D, b = 10, 10, 0, 120, 4
    ys = {}
    for polish in (1, 2):
        c = heff_case(L, N, tsz, D, 550, b, oracle=(polish == 1), precision=g.MIXED_BF16X3, mixed_polish=polish)
        ctx = c["ctx"]
        secs, info = ctx.tables(b)
        x = np.random.default_rng(9).normal(size=info["dim"])
        ys[polish] = ctx.apply_heff(b, x, precision=g.FP64)
        tm = ctx.timers()
        assert (tm["enlarge_tc_gflop"] > 0) == (polish == 2), tm
        if polish == 1:
            y_ref = c["He"].matvec(x)
            assert np.linalg.norm(ys[1] - y_ref) <= 1e-12 * np.linalg.norm(y_ref)
    assert np.linalg.norm(ys[2] - ys[1]) <= 1e-8 * np.linalg.norm(ys[1])
