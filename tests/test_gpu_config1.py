"""The smallest workload end to end (Eq. 3, Sec. II.B): L=10, N=10, 2S_z=0.

D=256: four full FP64 sweeps on the GPU from the same seeded MPS as the
oracle run stored in golden/config1.json (written by golden/make_config1.py
from the oracle only) give the oracle's Davidson energy at every step within
1e-9 Eh, and never go below the full-CI energy (variational, Eq. 3).
D=1024 is the full bond space at the central cut (sum_(a,b) C(5,a) C(5,b) =
1024), so the sweep reaches the full-CI energy (dimension 63504) within
1e-9 Eh; the mixed form (BF16x3 products, sliced anchors) reaches the FP64
result within 1e-6 Eh.
"""
import json
import os

import numpy as np
import pytest

import inputs
import paper_2412_04676_gb300 as g

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def golden():
    from paper_2412_04676_gb300 import build
    build.build()
    with open(os.path.join(HERE, "golden", "config1.json")) as f:
        return json.load(f)


def _run(gd, D, nsweeps, **kw):
    L, N, tsz = gd["L"], gd["N"], gd["tsz"]
    h, eri = inputs.make_integrals(L, gd["seed_integrals"])
    sites, dims = inputs.make_mps(L, N, tsz, D, gd["seed_mps"])
    c = g.Context(L, N, tsz, D=D, **kw)
    c.load_integrals(h, eri)
    c.import_mps(sites, [1] * L)
    st = c.sweep(nsweeps, D)
    e = c.step_energies()
    c.close()
    return st, e


def test_d256_four_sweeps_match_oracle_step_by_step(golden):
    st, e = _run(golden, golden["D"], golden["sweeps"], dav_tol=golden["dav_tol"])
    want = np.array(golden["step_energies"])
    assert e.shape == want.shape
    assert np.abs(e - want).max() <= 1e-9, np.abs(e - want).max()
    assert e.min() >= golden["e_fci"] - 1e-10
    # the last sweep cannot be above the first (variational decrease, Eq. 3)
    assert st[-1]["energy_last"] <= st[0]["energy_last"] + 1e-10


def test_d1024_full_bond_space_reaches_fci(golden):
    st, e = _run(golden, 1024, 2, dav_tol=1e-10)
    assert abs(e[-1] - golden["e_fci"]) <= 1e-9, (e[-1], golden["e_fci"])


def test_d1024_mixed_form_within_1e6_of_fp64(golden):
    _, e64 = _run(golden, 1024, 2, dav_tol=1e-10)
    _, em = _run(golden, 1024, 2, dav_tol=1e-8, precision=g.MIXED_BF16X3)
    assert abs(em[-1] - e64[-1]) <= 1e-6, (em[-1], e64[-1])
