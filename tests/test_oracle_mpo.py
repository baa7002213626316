"""Pins for oracle.mpo: the left/right split of Eq. 1 at every cut (Sec. II.B)."""
import numpy as np
import pytest

import inputs
from oracle import hamiltonian as H
from oracle import mpo as M


@pytest.mark.parametrize("L,seed", [(1, 3), (2, 4), (3, 5), (4, 6), (5, 7)])
def test_mpo_contracts_to_jordan_wigner_matrix(L, seed):
    # brute force: the product of all W[k] is the 4^L x 4^L matrix of Eq. 1
    h, eri = inputs.make_integrals(L, seed)
    mp = M.MPO(L, H.hamiltonian_terms(h, eri))
    Hd = M.mpo_to_dense(mp)
    Hj = H.jw_hamiltonian(h, eri).toarray()
    assert np.abs(Hd - Hj).max() < 1e-12 * max(1.0, np.abs(Hj).max())


def test_mpo_entries_conserve_quantum_numbers():
    # every nonzero W[k][a,c][s,t] moves (n, 2Sz) by dq_c - dq_a = q_s - q_t
    L = 6
    h, eri = inputs.make_integrals(L, 9)
    mp = M.MPO(L, H.hamiltonian_terms(h, eri))
    QS = np.array(inputs.QS)
    for k in range(L):
        for (a, c), W in mp.W[k].items():
            for s in range(4):
                for t in range(4):
                    if W[s, t] != 0.0:
                        assert np.array_equal(mp.dq[k + 1][c] - mp.dq[k][a], QS[s] - QS[t])
    assert mp.bond_dim(0) == 1 and mp.bond_dim(L) == 1


def test_site_order_sign():
    # a+_2 a_0 = - a_0 a+_2 (different orbitals anticommute); same-orbital order is kept
    s, o = M.site_order(((2, 0, 1), (0, 0, 0)))
    assert s == -1.0 and o == ((0, 0, 0), (2, 0, 1))
    s, o = M.site_order(((1, 0, 1), (1, 1, 1), (0, 1, 0), (0, 0, 0)))
    assert s == 1.0 and o == ((0, 1, 0), (0, 0, 0), (1, 0, 1), (1, 1, 1))
