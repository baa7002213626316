"""Writes config1.json: the oracle's DMRG energies for the smallest workload.

L=10 orbitals, N=10 electrons, 2S_z=0, D=256, integrals from seed 1001, the
random right-isometric start MPS from seed 1002 (both from ``inputs``); four
full sweeps (left-to-right over the cuts 0..L-3, right-to-left over L-2..1)
of the oracle's two-site DMRG (Sec. II.B, Eqs. 2-3) with Davidson tolerance
1e-10, the Davidson energy of every step in order, and the full-CI ground
energy of the same integrals (Eq. 3 over the whole (N, S_z) space, dimension
C(10,5)^2 = 63504).  Only ``oracle`` and ``inputs`` are called.

    python tests/golden/make_config1.py
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import inputs  # noqa: E402
from oracle import dmrg as R  # noqa: E402
from oracle import hamiltonian as H  # noqa: E402
from oracle import mpo as M  # noqa: E402

L, N, TSZ, D, SWEEPS, TOL = 10, 10, 0, 256, 4, 1e-10
SEED_INT, SEED_MPS = 1001, 1002


def main():
    t0 = time.time()
    h, eri = inputs.make_integrals(L, SEED_INT)
    sites, dims = inputs.make_mps(L, N, TSZ, D, SEED_MPS)
    mp = M.MPO(L, H.hamiltonian_terms(h, eri))
    dm = R.DMRG(mp, sites, dims, N, TSZ, D, tol=TOL)
    for _ in range(SWEEPS):
        dm.sweep()
    e_fci = H.fci_ground_energy(h, eri, N, TSZ)
    out = dict(L=L, N=N, tsz=TSZ, D=D, sweeps=SWEEPS, dav_tol=TOL, seed_integrals=SEED_INT, seed_mps=SEED_MPS,
               step_energies=[x["e"] for x in dm.log], step_resid=[x["resid"] for x in dm.log],
               step_trunc=[x["trunc"] for x in dm.log], e_fci=e_fci,
               note="written by tests/golden/make_config1.py from the oracle only",
               oracle_seconds=time.time() - t0)
    with open(os.path.join(HERE, "config1.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(f"E_last = {out['step_energies'][-1]:.12f}  E_FCI = {e_fci:.12f}  ({out['oracle_seconds']:.0f} s)")


if __name__ == "__main__":
    main()
