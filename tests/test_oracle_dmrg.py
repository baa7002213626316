"""Pins for oracle.dmrg: H_eff psi, Davidson, truncation and sweeps (Sec. II.B, Eqs. 2-3).

H_eff psi is pinned to its plain definition P^T H P psi evaluated in the Fock
space (Jordan-Wigner matrix for L <= 6, full-CI sigma vector for L = 8);
the sweep is pinned to full CI at full bond dimension and to the variational
bound of Eq. 3 below it.
"""
import numpy as np
import pytest

import inputs
from oracle import dmrg as R
from oracle import hamiltonian as H
from oracle import mpo as M


def _setup(L, N, tsz, D, seed, b):
    h, eri = inputs.make_integrals(L, seed)
    mp = M.MPO(L, H.hamiltonian_terms(h, eri))
    sites, dims = inputs.make_mps(L, N, tsz, D, seed + 1, n_left=b)
    psi4 = inputs.make_psi(dims, b, seed + 2)
    EL = R.build_left_envs(sites, dims, mp, b)[b]
    ER = R.build_right_envs(sites, dims, mp, b + 2, (N, tsz))[b + 2]
    He = R.Heff(EL, ER, dims, mp, b)
    return h, eri, mp, sites, dims, psi4, He


@pytest.mark.parametrize("b", [0, 1, 2, 3, 4])
def test_heff_equals_fock_projection_jw(b):
    L, N, tsz = 6, 6, 0
    h, eri, mp, sites, dims, psi4, He = _setup(L, N, tsz, 10, 40, b)
    y = He.to_blocks(He.apply(He.to_enlarged(psi4, None)))
    yf = R.heff_fock(H.jw_hamiltonian(h, eri), sites, dims, b, psi4, L)
    scale = max(np.abs(v).max() for v in yf.values())
    assert set(yf) <= set(y)
    for k in yf:
        assert np.abs(y[k] - yf[k]).max() <= 1e-12 * scale


def test_heff_equals_fock_projection_fci_sigma():
    L, N, tsz, b = 8, 7, 1, 3
    h, eri, mp, sites, dims, psi4, He = _setup(L, N, tsz, 20, 50, b)
    f = H.FCI(h, eri, N, tsz)
    y = He.to_blocks(He.apply(He.to_enlarged(psi4, None)))
    yf = R.heff_fock_fci(f, sites, dims, b, psi4, L)
    scale = max(np.abs(v).max() for v in yf.values())
    for k in yf:
        assert np.abs(y[k] - yf[k]).max() <= 1e-12 * scale


def test_heff_hermitian_and_davidson_matches_dense():
    L, N, tsz, b = 6, 6, 0, 2
    h, eri, mp, sites, dims, psi4, He = _setup(L, N, tsz, 10, 60, b)
    rng = np.random.default_rng(0)
    x, z = rng.normal(size=He.dim), rng.normal(size=He.dim)
    Hx, Hz = He.matvec(x), He.matvec(z)
    assert abs(z @ Hx - x @ Hz) <= 1e-12 * np.linalg.norm(Hx) * np.linalg.norm(z)
    Hd = np.array([He.matvec(e) for e in np.eye(He.dim)]).T
    assert np.allclose(np.diag(Hd), He.diagonal(), atol=1e-12)
    ev = np.linalg.eigvalsh(0.5 * (Hd + Hd.T))
    th, v, rn, nmv = R.davidson(He.matvec, He.diagonal(), rng.normal(size=He.dim), tol=1e-9)
    assert abs(th - ev[0]) < 1e-10 and rn <= 1e-9


def test_select_states_tie_rule_and_weight():
    ev = {(0, 0): np.array([0.5, 0.2]), (1, 1): np.array([0.2, 0.05]), (1, -1): np.array([0.05])}
    kept, w = R.select_states(ev, 3)
    # 0.5, 0.2, 0.2 fit; no tie straddles the cut
    assert kept == {(0, 0): 2, (1, 1): 1} and abs(w - 0.1) < 1e-15
    kept, w = R.select_states(ev, 2)
    # 0.2 and 0.2 straddle the cut at D = 2 -> cut moves down to 1
    assert kept == {(0, 0): 1} and abs(w - 0.5) < 1e-15
    kept, w = R.select_states({(0, 0): np.array([1.0, 1e-40])}, 5)
    assert kept == {(0, 0): 1}


def test_truncation_exact_when_not_truncating():
    rng = np.random.default_rng(3)
    psi = {(0, 0): rng.normal(size=(3, 5)), (1, 1): rng.normal(size=(4, 2))}
    nrm = np.sqrt(sum((x * x).sum() for x in psi.values()))
    psi = {k: v / nrm for k, v in psi.items()}
    U, C, w = R.truncate_left(psi, 100)
    for Q in psi:
        assert np.allclose(U[Q] @ C[Q], psi[Q], atol=1e-13)
        assert np.allclose(U[Q].T @ U[Q], np.eye(U[Q].shape[1]), atol=1e-13)
    assert w < 1e-14
    V, C, w = R.truncate_right(psi, 4)
    ev = np.sort(np.concatenate([np.linalg.svd(x, compute_uv=False) ** 2 for x in psi.values()]))[::-1]
    assert abs(w - ev[4:].sum()) < 1e-13


def test_dmrg_full_bond_dimension_reproduces_fci():
    L, N, tsz = 6, 6, 0
    h, eri = inputs.make_integrals(L, 71)
    mp = M.MPO(L, H.hamiltonian_terms(h, eri))
    sites, dims = inputs.make_mps(L, N, tsz, 64, 72)
    d = R.DMRG(mp, sites, dims, N, tsz, 64, tol=1e-9)
    e_last = [d.sweep()[0] for _ in range(2)][-1]
    assert abs(e_last - H.fci_ground_energy(h, eri, N, tsz)) < 1e-10


def test_dmrg_truncated_is_variational_and_decreasing():
    L, N, tsz = 7, 6, 2
    h, eri = inputs.make_integrals(L, 81)
    mp = M.MPO(L, H.hamiltonian_terms(h, eri))
    sites, dims = inputs.make_mps(L, N, tsz, 6, 82)
    d = R.DMRG(mp, sites, dims, N, tsz, 6, tol=1e-9)
    e_fci = H.fci_ground_energy(h, eri, N, tsz)
    es = [d.sweep()[0] for _ in range(3)]
    assert all(e >= e_fci - 1e-10 for e in es)
    assert es[1] <= es[0] + 1e-10 and es[2] <= es[1] + 1e-10
    assert any(x["trunc"] > 0 for x in d.log)
