"""Pins for oracle.hamiltonian: Eq. 1 of arXiv:2412.04676 (Sec. II.A) and its exact solutions.

Each check fixes the oracle against something other than itself: a second,
independent construction (Jordan-Wigner Kronecker products vs. determinant
strings), closed forms, and a library eigensolver.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as sla

import inputs
from oracle import hamiltonian as H


def test_integral_symmetry_and_psd():
    h, eri = inputs.make_integrals(7, 123)
    assert np.allclose(h, h.T)
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (1, 0, 3, 2), (3, 2, 1, 0)]:
        assert np.allclose(eri, eri.transpose(perm))
    M = eri.reshape(49, 49)
    assert np.linalg.eigvalsh(M).min() > -1e-10
    assert np.all(np.diff(np.diag(h)) >= 0)  # ascending orbital energies


@pytest.mark.parametrize("L,N,tsz,seed", [(3, 3, 1, 1), (4, 4, 0, 2), (4, 3, 1, 3), (5, 4, 2, 4), (5, 6, 0, 5)])
def test_fci_matches_jordan_wigner(L, N, tsz, seed):
    h, eri = inputs.make_integrals(L, seed)
    assert abs(H.fci_ground_energy(h, eri, N, tsz) - H.jw_ground_energy(h, eri, N, tsz)) < 1e-10


def test_fci_sigma_equals_jw_matrix_elementwise():
    # the whole FCI matrix, not just its lowest eigenvalue
    L, N, tsz = 4, 4, 0
    h, eri = inputs.make_integrals(L, 31)
    f = H.FCI(h, eri, N, tsz)
    dim = f.shape[0] * f.shape[1]
    Hf = np.array([f.matvec(e) for e in np.eye(dim)]).T
    Hj = H.jw_hamiltonian(h, eri)
    n, t = H.occupation_labels(L)
    idx = np.where((n == N) & (t == tsz))[0]
    assert np.allclose(np.linalg.eigvalsh(Hf), np.linalg.eigvalsh(Hj[idx][:, idx].toarray()), atol=1e-11)
    assert np.allclose(Hf, Hf.T, atol=1e-12)


def test_noninteracting_closed_form():
    # V = 0: E = sum of the lowest N_up eigenvalues of h + lowest N_dn
    h, eri = inputs.make_integrals(6, 77)
    ev = np.linalg.eigvalsh(h)
    for N, tsz in [(6, 0), (5, 1), (4, 2)]:
        na, nb = (N + tsz) // 2, (N - tsz) // 2
        e = H.fci_ground_energy(h, np.zeros_like(eri), N, tsz)
        assert abs(e - (ev[:na].sum() + ev[:nb].sum())) < 1e-11


def test_one_orbital_two_electrons():
    h = np.array([[-0.8]])
    eri = np.array([[[[0.45]]]])
    assert abs(H.fci_ground_energy(h, eri, 2, 0) - (2 * -0.8 + 0.45)) < 1e-14
    assert abs(H.jw_ground_energy(h, eri, 2, 0) - (2 * -0.8 + 0.45)) < 1e-14


def test_two_orbitals_two_electrons_closed_form():
    # S_z = 0 space of 2 electrons in 2 orbitals: three singlets + the m=0 triplet
    h, eri = inputs.make_integrals(2, 5)
    J, K = eri[0, 0, 1, 1], eri[0, 1, 0, 1]
    s2 = np.sqrt(2.0)
    Hs = np.array([
        [2 * h[0, 0] + eri[0, 0, 0, 0], K, s2 * (h[0, 1] + eri[0, 0, 0, 1])],
        [K, 2 * h[1, 1] + eri[1, 1, 1, 1], s2 * (h[0, 1] + eri[1, 1, 0, 1])],
        [s2 * (h[0, 1] + eri[0, 0, 0, 1]), s2 * (h[0, 1] + eri[1, 1, 0, 1]), h[0, 0] + h[1, 1] + J + K],
    ])
    expect = np.sort(np.concatenate([np.linalg.eigvalsh(Hs), [h[0, 0] + h[1, 1] + J - K]]))
    f = H.FCI(h, eri, 2, 0)
    Hf = np.array([f.matvec(e) for e in np.eye(4)]).T
    assert np.allclose(np.sort(np.linalg.eigvalsh(Hf)), expect, atol=1e-13)


def test_lanczos_matches_library_eigsh():
    h, eri = inputs.make_integrals(6, 8)
    f = H.FCI(h, eri, 6, 0)
    dim = f.shape[0] * f.shape[1]
    e, x = H.lanczos_lowest(f.matvec, dim)
    op = sla.LinearOperator((dim, dim), matvec=f.matvec, dtype=np.float64)
    ref = sla.eigsh(op, k=1, which="SA", tol=1e-13)[0][0]
    assert abs(e - ref) < 1e-10
    assert np.linalg.norm(f.matvec(x) - e * x) < 1e-6
