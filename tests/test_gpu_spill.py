"""The bounded host store: spill to a file and read back (Sec. III.A, III.B.4).

With host_store_bytes set, at most that many bytes of packed environments
stay in pinned host memory; the least recently used go to a spill file
through an IO thread and are read back before a step unpacks them.  Packages
are self-contained (Sec. III.B.3), so a spilled environment comes back byte
for byte, and whole sweeps give exactly the energies of an unbounded store.
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


def _ctx(budget, L=8, N=8, D=40, n_left=0, seed=900):
    h, eri = inputs.make_integrals(L, seed)
    sites, dims = inputs.make_mps(L, N, 0, D, seed + 1, n_left=n_left)
    c = g.Context(L, N, 0, D=D, offload=True, host_store_bytes=budget, dav_tol=1e-10)
    c.load_integrals(h, eri)
    c.import_mps(sites, [0] * n_left + [1] * (L - n_left))
    return c


def test_spilled_sweep_equals_unbounded_store():
    out = {}
    for budget in (0, 64 << 10):
        c = _ctx(budget)
        c.sweep(2, 40)
        out[budget] = (c.step_energies(), c.timers())
        c.close()
    assert np.array_equal(out[0][0], out[64 << 10][0])
    t = out[64 << 10][1]
    assert t["spill_gbytes"] > 0 and t["restore_gbytes"] > 0
    assert out[0][1]["spill_gbytes"] == 0


def test_spilled_environment_round_trip_is_byte_exact():
    b = 2
    c = _ctx(1, n_left=b, seed=910)   # every save beyond the first goes to the file
    c.build_envs(b)
    c.step(b, 1, 40)
    before = c.env_export(0, b + 1)
    c.step(b + 1, 1, 40)              # releases it from the device; later saves spill it
    c.step(b + 2, 1, 40)
    after = c.env_export(0, b + 1)    # read back from the spill file, unpacked, checksums verified
    t = c.timers()
    assert t["spill_gbytes"] > 0 and t["restore_gbytes"] > 0
    assert after.tobytes() == before.tobytes()
    c.close()
