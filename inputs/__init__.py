"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This module only draws random numbers and shapes them into the objects both
sides consume: one- and two-electron integrals, a random matrix product state
(MPS) with U(1)xU(1) symmetry sectors, a random two-site wavefunction, and
random block-sparse environments for the pack/unpack tests.  It holds none of
the method's arithmetic (no Hamiltonian, no environment contraction, no
effective Hamiltonian, no Davidson, no truncation).

Conventions used by every consumer
----------------------------------
* Spatial orbitals (sites) are numbered 0..L-1 in the order of ascending
  orbital energy h_ii (no reordering).
* Local basis of a site, index s: 0 = |0>, 1 = |up>, 2 = |dn>,
  3 = |updn> = c+_up c+_dn |0>.
* Quantum numbers are pairs q = (n, tsz) with tsz = n_up - n_dn (twice S_z).
  A bond label is counted from the left: the bond after site k carries the
  particle number and 2S_z of sites 0..k.
* A site tensor is a dict {(q_left, s): block} whose block has
  rows = dim(q_left) on the left bond and cols = dim(q_left + q_s) on the
  right bond (row-major, float64).

Integral recipe (stand-in for the FeMoco integrals of Sec. IV, which are not
available): rng = numpy.random.default_rng(seed); orbital energies
e = sort(rng.uniform(-2, 1, L)) on the diagonal of h; the strict upper
triangle of h drawn row-major from N(0, 0.1) (second argument = standard
deviation) and mirrored; for P = 0..19 the upper triangle including the
diagonal of B^P drawn row-major from N(0, 0.3) and mirrored;
(ij|kl) = sum_P B^P_ij B^P_kl, which has the 8-fold permutational symmetry
and is positive semidefinite as a matrix over pairs (ij),(kl).
"""
from __future__ import annotations

from math import comb

import numpy as np

QS = ((0, 0), (1, 1), (1, -1), (2, 0))  # (n, tsz) of the four local states

# Workloads: (L, N, tsz, D, seed) for the five configurations.
CONFIGS = {
    1: dict(L=10, N=10, tsz=0, D=256, seed=1001),
    2: dict(L=30, N=30, tsz=0, D=1024, seed=1002),
    3: dict(L=54, N=54, tsz=0, D=2048, seed=1003),
    4: dict(L=76, N=113, tsz=1, D=4096, seed=1004),
    5: dict(L=76, N=113, tsz=1, D=8192, seed=1005),
}


def make_integrals(L: int, seed: int, naux: int = 20):
    """Return (h, eri) with h (L, L) symmetric and eri (L, L, L, L) chemist (ij|kl)."""
    rng = np.random.default_rng(seed)
    e = np.sort(rng.uniform(-2.0, 1.0, L))
    h = np.diag(e).astype(np.float64)
    iu = np.triu_indices(L, k=1)
    off = rng.normal(0.0, 0.1, size=len(iu[0]))
    h[iu] = off
    h[(iu[1], iu[0])] = off
    B = np.zeros((naux, L, L))
    iu0 = np.triu_indices(L, k=0)
    for P in range(naux):
        v = rng.normal(0.0, 0.3, size=len(iu0[0]))
        B[P][iu0] = v
        B[P][(iu0[1], iu0[0])] = v
    eri = np.einsum("pij,pkl->ijkl", B, B)
    return h, eri


def add_q(a, b):
    return (a[0] + b[0], a[1] + b[1])


def sub_q(a, b):
    return (a[0] - b[0], a[1] - b[1])


def bond_dims(L: int, N: int, tsz: int, D: int):
    """Sector dimensions of every bond 0..L of a random initial MPS.

    Each allowed sector q of bond k (left block = sites 0..k-1) gets
    min(full_left, full_right, round(D * w_q / sum w)) states with
    w_q = full_left(q) * full_right(q), the number of determinants with that
    split (free-fermion multiplicity).  Sectors that round to zero are
    dropped.  Two passes then make every site map feasible for both left- and
    right-isometries.
    """
    na, nb = (N + tsz) // 2, (N - tsz) // 2
    assert na + nb == N and na - nb == tsz and 0 <= nb <= na <= L
    dims = []
    for k in range(L + 1):
        cand = {}
        for a in range(max(0, na - (L - k)), min(k, na) + 1):
            for b in range(max(0, nb - (L - k)), min(k, nb) + 1):
                fl = comb(k, a) * comb(k, b)
                fr = comb(L - k, na - a) * comb(L - k, nb - b)
                cand[(a + b, a - b)] = (fl, fr)
        tot = sum(fl * fr for fl, fr in cand.values())
        d = {}
        for q, (fl, fr) in cand.items():
            x = min(fl, fr, int(round(D * fl * fr / tot)))
            if x > 0:
                d[q] = x
        dims.append(d)
    for _ in range(4):
        for k in range(1, L + 1):  # left feasibility
            for q in list(dims[k]):
                cap = sum(dims[k - 1].get(sub_q(q, qs), 0) for qs in QS)
                dims[k][q] = min(dims[k][q], cap)
                if dims[k][q] == 0:
                    del dims[k][q]
        for k in range(L, 0, -1):  # right feasibility
            for q in list(dims[k - 1]):
                cap = sum(dims[k].get(add_q(q, qs), 0) for qs in QS)
                dims[k - 1][q] = min(dims[k - 1][q], cap)
                if dims[k - 1][q] == 0:
                    del dims[k - 1][q]
    return dims


def _left_iso(dl, dr, rng):
    """Random left-isometric site tensor between bond dims dl -> dr."""
    site = {}
    for q, m in dr.items():
        rows = [(qs_i, dl[sub_q(q, qs)]) for qs_i, qs in enumerate(QS) if sub_q(q, qs) in dl]
        tot = sum(r for _, r in rows)
        M = rng.normal(size=(tot, m))
        Q, _ = np.linalg.qr(M)
        off = 0
        for s, r in rows:
            site[(sub_q(q, QS[s]), s)] = np.ascontiguousarray(Q[off:off + r, :m])
            off += r
    return site


def _right_iso(dl, dr, rng):
    """Random right-isometric site tensor between bond dims dl -> dr."""
    site = {}
    for q, m in dl.items():
        cols = [(s, dr[add_q(q, qs)]) for s, qs in enumerate(QS) if add_q(q, qs) in dr]
        tot = sum(c for _, c in cols)
        M = rng.normal(size=(tot, m))
        Q, _ = np.linalg.qr(M)
        R = Q[:, :m].T  # m x tot, orthonormal rows
        off = 0
        for s, c in cols:
            site[(q, s)] = np.ascontiguousarray(R[:, off:off + c])
            off += c
    return site


def make_mps(L: int, N: int, tsz: int, D: int, seed: int, n_left: int = 0):
    """Random MPS: sites 0..n_left-1 left-isometric, the rest right-isometric.

    Returns (sites, dims) where dims = bond_dims(...) and sites[k] is the dict
    tensor of site k.  With n_left = 0 every site is right-isometric and the
    state has unit norm.
    """
    rng = np.random.default_rng(seed)
    dims = bond_dims(L, N, tsz, D)
    sites = []
    for k in range(L):
        if k < n_left:
            sites.append(_left_iso(dims[k], dims[k + 1], rng))
        else:
            sites.append(_right_iso(dims[k], dims[k + 1], rng))
    return sites, dims


def make_psi(dims, b: int, seed: int):
    """Random normalised two-site wavefunction on sites (b, b+1).

    Keys are (q_left, s1, s2) with q_left a sector of bond b (left of site b);
    the block has rows dim_b(q_left), cols dim_{b+2}(q_left + q_s1 + q_s2).
    """
    rng = np.random.default_rng(seed)
    psi = {}
    for q, m in dims[b].items():
        for s1 in range(4):
            for s2 in range(4):
                qr = add_q(add_q(q, QS[s1]), QS[s2])
                if qr in dims[b + 2]:
                    psi[(q, s1, s2)] = rng.normal(size=(m, dims[b + 2][qr]))
    nrm = np.sqrt(sum(float(np.sum(x * x)) for x in psi.values()))
    for k in psi:
        psi[k] /= nrm
    return psi


def make_env_blocks(n_classes: int, seed: int, max_dim: int = 40, max_layers: int = 12,
                    empty_every: int = 0):
    """Random block-sparse environment for the pack/unpack tests.

    Returns a list of classes; each class is a dict with 'dq' (n, tsz), a
    list 'layers' of MPO state ids and a list 'blocks' of
    (q_out, q_in, rows, cols, data) with data of shape (n_layers, rows, cols).
    Sizes are drawn so that empty and 1x1 blocks occur.
    """
    rng = np.random.default_rng(seed)
    classes = []
    wid = 0
    for c in range(n_classes):
        nl = int(rng.integers(1, max_layers + 1))
        dq = (int(rng.integers(-2, 3)), int(rng.integers(-2, 3)))
        layers = list(range(wid, wid + nl))
        wid += nl
        blocks = []
        nb = int(rng.integers(0, 9))
        for j in range(nb):
            r = int(rng.integers(0, max_dim + 1)) if rng.random() < 0.8 else 1
            cc = int(rng.integers(0, max_dim + 1)) if rng.random() < 0.8 else 1
            if empty_every and j % empty_every == 0:
                r = 0
            qin = (int(rng.integers(0, 20)), int(rng.integers(-6, 7)))
            qout = add_q(qin, dq)
            data = rng.normal(size=(nl, r, cc))
            blocks.append((qout, qin, r, cc, data))
        classes.append(dict(dq=dq, layers=layers, blocks=blocks))
    return classes
