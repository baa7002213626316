"""Failure detection made on the host (no device fault, trap or hang).

Each case switches on one host-side fault through gbd_config.fault_inject and
checks the status the C-ABI returns: a refused pinned allocation of the
offload store (GBD_ERR_HOST_OOM), IO events that never report completion
(bounded waits run out: GBD_ERR_TIMEOUT), a corrupted host copy of an
offloaded environment (package checksum, Sec. III.B.3: GBD_ERR_CORRUPT), and
a Davidson that reaches its product limit (GBD_WARN_NOT_CONVERGED).
"""
import pytest

import inputs
import paper_2412_04676_gb300 as g

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2412_04676_gb300 import build
    build.build()


def _sweep_ctx(fault, io_timeout_ms=120000):
    L, N, D = 6, 6, 16
    h, eri = inputs.make_integrals(L, 41)
    sites, dims = inputs.make_mps(L, N, 0, D, 42)
    c = g.Context(L, N, 0, D=D, offload=True, fault_inject=fault, io_timeout_ms=io_timeout_ms)
    c.load_integrals(h, eri)
    c.import_mps(sites, [1] * L)
    return c


def test_refused_pinned_allocation_gives_host_oom():
    c = _sweep_ctx(g.FAULT_PINNED_ALLOC)
    with pytest.raises(g.GbdError) as e:
        c.sweep(1, 16)
    assert e.value.code == -3
    c.close()


def test_io_wait_runs_out_gives_timeout():
    c = _sweep_ctx(g.FAULT_IO_NEVER_READY, io_timeout_ms=1)
    with pytest.raises(g.GbdError) as e:
        c.sweep(1, 16)
    assert e.value.code == -5
    c.close()


def test_corrupted_host_copy_is_caught_on_load():
    c = _sweep_ctx(g.FAULT_CORRUPT_HOST_COPY)
    with pytest.raises(g.GbdError) as e:
        c.sweep(1, 16)
    assert e.value.code == -6
    c.close()


def test_without_faults_the_same_sweep_succeeds():
    c = _sweep_ctx(0)
    st = c.sweep(1, 16)
    assert st[0]["bytes_packed"] > 0
    c.close()


def test_davidson_product_limit_is_a_warning():
    L, N, D, b = 8, 8, 24, 3
    h, eri = inputs.make_integrals(L, 43)
    sites, dims = inputs.make_mps(L, N, 0, D, 44, n_left=b)
    c = g.Context(L, N, 0, D=D, dav_tol=1e-14, dav_max_matvec=2)
    c.load_integrals(h, eri)
    c.import_mps(sites, [0] * b + [1] * (L - b))
    c.build_envs(b)
    e, _, st, rc = c.davidson(b)
    assert rc == g.WARN_NOT_CONVERGED and st["matvecs"] == 2
    s = c.step(b, 1, D)
    assert s["dav_status"] == g.WARN_NOT_CONVERGED
    c.close()


def test_mixed_davidson_reports_its_precision_floor():
    # a tolerance below what the anchor products can resolve: once an anchor
    # no longer cuts the exact residual by a fifth the mixed Davidson stops and says so
    # (the result is its best anchored pair)
    L, N, D, b = 8, 8, 24, 3
    h, eri = inputs.make_integrals(L, 45)
    sites, dims = inputs.make_mps(L, N, 0, D, 46, n_left=b)
    c = g.Context(L, N, 0, D=D, precision=g.MIXED_BF16X3, dav_tol=1e-15, dav_max_matvec=2000)
    c.load_integrals(h, eri)
    c.import_mps(sites, [0] * b + [1] * (L - b))
    c.build_envs(b)
    e, _, st, rc = c.davidson(b)
    assert rc == g.WARN_PRECISION_FLOOR and st["resid"] > 1e-15 and st["matvecs"] < 2000
    ref = g.Context(L, N, 0, D=D, dav_tol=1e-11)
    ref.load_integrals(h, eri)
    ref.import_mps(sites, [0] * b + [1] * (L - b))
    ref.build_envs(b)
    e64, _, _, rc64 = ref.davidson(b)
    assert rc64 == 0 and abs(e - e64) < 1e-8
    c.close()
    ref.close()
