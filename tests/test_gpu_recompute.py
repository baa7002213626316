"""Environment recomputation instead of IO (Sec. IV, the on-the-fly
alternative to storing environments).

With env_recompute = k only environments at cuts divisible by k (and the
chain ends) go to the pinned host store; the others are dropped after use
and rebuilt when a step needs them, from the nearest stored one, by the same
enlargement and renormalisation the sweep uses (Sec. II.B steps 1 and 3).
In the FP64 form the rebuilt environments are the ones the sweep made, so
whole sweeps give the same energies as with every environment stored, with
fewer bytes moved to the host.
"""
import numpy as np
import pytest

import inputs
import paper_2412_04676_gb300 as g

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2412_04676_gb300 import build
    build.build()


def _sweeps(prec, recompute, L=10, N=10, D=40, n=2, tol=1e-10):
    h, eri = inputs.make_integrals(L, 800)
    sites, dims = inputs.make_mps(L, N, 0, D, 801)
    c = g.Context(L, N, 0, D=D, precision=prec, offload=True, env_recompute=recompute, dav_tol=tol)
    c.load_integrals(h, eri)
    c.import_mps(sites, [1] * L)
    st = c.sweep(n, D)
    out = (c.step_energies(), c.io_stats(), c.timers(), st)
    c.close()
    return out


def test_recomputed_environments_give_the_stored_sweep():
    e0, io0, t0, _ = _sweeps(g.FP64, 0)
    e3, io3, t3, st = _sweeps(g.FP64, 3)
    assert e0.shape == e3.shape
    assert np.abs(e3 - e0).max() <= 1e-12, np.abs(e3 - e0).max()
    assert t3["recompute_n"] > 0 and t0["recompute_n"] == 0
    assert io3["bytes_d2h"] < io0["bytes_d2h"]
    assert st[-1]["energy_last"] <= st[0]["energy_last"] + 1e-10


def test_recompute_in_the_mixed_form():
    # the mixed form renormalises on the sliced tensor-core planes inside a
    # step and in FP64 when it recomputes: energies agree far inside 1e-6 Eh
    e0, _, _, _ = _sweeps(g.MIXED_BF16X3, 0, tol=1e-8)
    e2, _, t2, _ = _sweeps(g.MIXED_BF16X3, 2, tol=1e-8)
    assert t2["recompute_n"] > 0
    assert abs(e2[-1] - e0[-1]) <= 1e-7
