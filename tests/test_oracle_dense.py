"""Dense, unsymmetrised check of the oracle's block-sparse H_eff product
(Sec. II.B step 2): every operator layer of both enlarged blocks is written
out as a full matrix over all symmetry sectors (zeros off-sector), psi as a
full matrix with only three sectors non-zero, and sum_c O^L_c Psi (O^R_c)^T
is evaluated with no sector bookkeeping.  The block-sparse product must agree
on every sector it produces, and the dense result must vanish on every block
that breaks (N, 2S_z) conservation.  This pins the block pairing, the layer
intersection and the sector offsets; the formula itself is pinned by the
Fock-space projection tests.
"""
import numpy as np
import pytest

import inputs
from oracle import dmrg as R
from oracle import hamiltonian as H
from oracle import mpo as M


def _offsets(basis):
    keys = sorted(basis)
    off, o = {}, 0
    for q in keys:
        off[q] = o
        o += basis[q][1]
    return off, o


def _dense_layers(O, basis):
    off, n = _offsets(basis)
    layers = {}
    for (Q, Q2), (C, blk) in O.items():
        for c, b in zip(C, blk):
            A = layers.setdefault(int(c), np.zeros((n, n)))
            A[off[Q]:off[Q] + b.shape[0], off[Q2]:off[Q2] + b.shape[1]] += b
    return layers, off, n


@pytest.mark.parametrize("L,N,tsz,D,seed,b", [(8, 8, 0, 40, 610, 3), (8, 7, 1, 30, 611, 2), (10, 10, 0, 60, 612, 4)])
def test_block_sparse_product_matches_dense(L, N, tsz, D, seed, b):
    h, eri = inputs.make_integrals(L, seed)
    mp = M.MPO(L, H.hamiltonian_terms(h, eri))
    sites, dims = inputs.make_mps(L, N, tsz, D, seed + 1, n_left=b)
    EL = R.build_left_envs(sites, dims, mp, b)[b]
    ER = R.build_right_envs(sites, dims, mp, b + 2, (N, tsz))[b + 2]
    He = R.Heff(EL, ER, dims, mp, b)
    # the three largest sectors of psi non-zero
    rng = np.random.default_rng(seed)
    big = sorted(He.shape, key=lambda Q: -He.shape[Q][0] * He.shape[Q][1])[:3]
    psi = {Q: (rng.normal(size=He.shape[Q]) if Q in big else np.zeros(He.shape[Q])) for Q in He.shape}
    y = He.apply(psi)
    AL, offL, nL = _dense_layers(He.OL, He.bL)
    AR, offR, nR = _dense_layers(He.OR, He.bR)
    P = np.zeros((nL, nR))
    for Q in He.shape:
        P[offL[Q]:offL[Q] + He.shape[Q][0], offR[Q]:offR[Q] + He.shape[Q][1]] = psi[Q]
    Y = np.zeros((nL, nR))
    for c in set(AL) & set(AR):
        Y += AL[c] @ P @ AR[c].T
    scale = np.abs(Y).max()
    assert scale > 0
    mask = np.zeros_like(Y, dtype=bool)
    for Q, (a, bb) in He.shape.items():
        blk = Y[offL[Q]:offL[Q] + a, offR[Q]:offR[Q] + bb]
        assert np.abs(blk - y[Q]).max() <= 1e-12 * scale
        mask[offL[Q]:offL[Q] + a, offR[Q]:offR[Q] + bb] = True
    # nothing outside the (N, 2S_z)-conserving sector blocks
    assert np.abs(Y[~mask]).max(initial=0.0) <= 1e-12 * scale
