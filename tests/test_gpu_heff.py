"""GPU parity of the hot path H_eff psi (Sec. II.B step 2, Eqs. 2-3) against the oracle.

Both sides get the same seeded integrals, MPS and two-site vector; the library
builds its environments on the GPU (enlargement + renormalisation) and applies
H_eff through the C-ABI.  FP64 tolerance: 1e-12 relative to max|y| (the
product sums O(10^3) terms of size ~|y|, so rounding differences stay near
1e-14 relative; 1e-12 leaves two orders of margin).
"""
import numpy as np
import pytest

from gpu_common import build_lib, heff_case

pytestmark = pytest.mark.gpu
TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def built():
    build_lib()


@pytest.mark.parametrize("L,N,tsz,D,seed,b", [
    (6, 6, 0, 16, 100, 0), (6, 6, 0, 16, 101, 2), (6, 6, 0, 16, 102, 4),
    (8, 7, 1, 40, 103, 3), (8, 8, 2, 30, 104, 5), (10, 10, 0, 64, 105, 4),
])
def test_heff_matches_oracle(L, N, tsz, D, seed, b):
    c = heff_case(L, N, tsz, D, seed, b)
    ctx, He = c["ctx"], c["He"]
    secs, info = ctx.tables(b)
    assert info["dim"] == He.dim
    assert [s["q"] for s in secs] == [tuple(q) for q in He.sectors]
    x = He.flatten(He.to_enlarged(c["psi4"], None))
    y_ref = He.matvec(x)
    y = ctx.apply_heff(b, x)
    scale = np.abs(y_ref).max()
    assert np.abs(y - y_ref).max() <= TOL * scale
    d_ref = He.diagonal()
    d = ctx.heff_diagonal(b, He.dim)
    assert np.abs(d - d_ref).max() <= TOL * max(1.0, np.abs(d_ref).max())


def test_heff_ragged_and_large_sectors_span_tiles():
    # D large enough that sector blocks exceed one 64x64 tile with ragged edges
    L, N, tsz, D, b = 10, 9, 1, 200, 4
    c = heff_case(L, N, tsz, D, 107, b)
    ctx, He = c["ctx"], c["He"]
    secs, info = ctx.tables(b)
    assert max(s["rows"] for s in secs) > 64 and any(s["rows"] % 64 for s in secs)
    rng = np.random.default_rng(3)
    for _ in range(2):
        x = rng.normal(size=He.dim)
        y_ref = He.matvec(x)
        y = ctx.apply_heff(b, x)
        assert np.abs(y - y_ref).max() <= TOL * np.abs(y_ref).max()


def test_heff_hermitian_full_size_l30_d1024():
    # L=30, N=30, D=1024 at the mid-chain cut: properties that hold at any size
    L, N, tsz, D, b = 30, 30, 0, 1024, 14
    c = heff_case(L, N, tsz, D, 1002, b, oracle=False)
    ctx = c["ctx"]
    secs, info = ctx.tables(b)
    rng = np.random.default_rng(0)
    x, z = rng.normal(size=info["dim"]), rng.normal(size=info["dim"])
    Hx, Hz = ctx.apply_heff(b, x), ctx.apply_heff(b, z)
    assert abs(z @ Hx - x @ Hz) <= 1e-11 * np.linalg.norm(Hx) * np.linalg.norm(z)
    # linearity
    H2 = ctx.apply_heff(b, 2.0 * x - 3.0 * z)
    assert np.abs(H2 - (2 * Hx - 3 * Hz)).max() <= 1e-11 * np.abs(H2).max()
    assert info["n_terms"] > 1000 and info["useful_flops"] > 1e10


def test_per_block_launches_give_the_batched_result():
    # the comparison form: every sector block GEMM task in its own launch
    # (same kernel, same tiles) is bitwise the grouped product
    import paper_2412_04676_gb300 as g
    L, N, tsz, D, b = 10, 10, 0, 120, 4
    c = heff_case(L, N, tsz, D, 108, b)
    ctx, He = c["ctx"], c["He"]
    x = He.flatten(He.to_enlarged(c["psi4"], None))
    y = ctx.apply_heff(b, x, precision=g.FP64)
    n0 = g.launch_count()
    yb = ctx.apply_heff(b, x, precision=g.FP64_PER_BLOCK)
    n1 = g.launch_count()
    assert np.array_equal(y, yb)
    secs, info = ctx.tables(b)
    assert n1 - n0 > len(secs)          # at least one launch per output sector
    t = ctx.timers()
    assert t["products_fp64_per_block_n"] == 1 and t["products_fp64_per_block_ms"] > 0
