"""Eq. 1 split at every cut of the chain: the left/right operator sets of Sec. II.B.

A two-site DMRG step (Sec. II.B, Fig. 3a) needs, for every cut between a
left block and a right block, operator sets O^L_w and O^R_w with
H = sum_w O^L_w (x) O^R_w.  This module builds them directly from the terms
of Eq. 1, written in Jordan-Wigner form so that the Kronecker structure is
plain (bosonic):

* every term is put in site order (a stable sort by orbital; the sign is the
  parity of the permutation, since operators on different orbitals
  anticommute);
* the factor on orbital y is (the operators on y, in order) times
  P_y^(number of operators on orbitals > y), P = diag(1,-1,-1,1);
* the state of a term at cut k is 'I' before its first operator, 'F' after
  its last, ('P', placed operators) while at most two are placed (a normal
  operator of the left block) and ('S', remaining operators) once three are
  placed (a complementary operator: the coefficient is folded in when the
  term enters it, so terms that share the remaining operator are summed).

W[k] maps the states of cut k (left of orbital k) to those of cut k+1 with
a 4x4 matrix per pair.  The product W[0] W[1] ... W[L-1] (Kronecker in the
physical indices) is Eq. 1; ``mpo_to_dense`` checks that against the
Jordan-Wigner matrix.  This is the oracle's own construction: it has no
switch to complementary pairs, so its bond dimension grows as O(k^2).
"""
from __future__ import annotations

from collections import defaultdict

import numpy as np
import scipy.sparse as sp

from .hamiltonian import UP, local_ops


def _charge(spin, dag):
    sz = 1 if spin == UP else -1
    return (1, sz) if dag else (-1, -sz)


def site_order(ops):
    """Stable sort of ops by orbital; returns (sign, ordered ops)."""
    idx = sorted(range(len(ops)), key=lambda i: ops[i][0])
    inv = 0
    for a in range(len(idx)):
        for b in range(a + 1, len(idx)):
            if idx[a] > idx[b]:
                inv += 1
    return (-1.0) ** inv, tuple(ops[i] for i in idx)


class MPO:
    """Left/right operator sets of Eq. 1 for every cut 0..L.

    Attributes
    ----------
    states[k] : list of state keys alive at cut k (cut k = left of orbital k)
    dq[k]     : array (n_k, 2) of the (n, tsz) change made by the left part
    W[k]      : dict {(i, j): 4x4} with i a state at cut k, j at cut k+1
    """

    def __init__(self, L, terms):
        cu, cd, P = local_ops()
        loc = {(UP, 1): cu, (1 - UP, 1): cd, (UP, 0): cu.T, (1 - UP, 0): cd.T}
        self.L = L
        edges = [dict() for _ in range(L)]       # keyed by state keys
        lo = defaultdict(lambda: L + 1)           # first cut a key is alive
        hi = defaultdict(lambda: -1)              # last cut a key is alive
        rem_par = {}
        for coef, ops in terms:
            sign, ordered = site_order(ops)
            m = len(ordered)
            groups = []
            for op in ordered:
                if groups and groups[-1][0] == op[0]:
                    groups[-1][1].append(op)
                else:
                    groups.append((op[0], [op]))
            prev = ("I",)
            prev_cut = 0
            placed = 0
            for orb, gops in groups:
                lo[prev] = min(lo[prev], prev_cut)
                hi[prev] = max(hi[prev], orb)
                placed += len(gops)
                rem = m - placed
                M = np.eye(4)
                for (_, s, d) in gops:
                    M = M @ loc[(s, d)]
                if rem % 2:
                    M = M @ P
                if rem == 0:
                    new = ("F",)
                elif placed <= 2:
                    new = ("P", ordered[:placed])
                else:
                    new = ("S", ordered[placed:])
                rem_par[new] = rem % 2
                e = (prev, new)
                if new[0] in ("S", "F") and prev[0] in ("I", "P"):
                    edges[orb][e] = edges[orb].get(e, 0.0) + coef * sign * M
                else:
                    edges[orb][e] = M
                prev = new
                prev_cut = orb + 1
            lo[prev] = min(lo[prev], prev_cut)
            hi[prev] = L
        rem_par[("I",)] = 0
        rem_par[("F",)] = 0
        # pass-through: a state alive at cuts k and k+1 crosses orbital k
        for key in list(lo.keys()):
            for k in range(lo[key], hi[key]):
                M = P if rem_par[key] else np.eye(4)
                edges[k].setdefault((key, key), M)
        self.states = []
        for c in range(L + 1):
            alive = [key for key in lo if lo[key] <= c <= hi[key]]
            alive.sort(key=_sort_key)
            self.states.append(alive)
        index = [{key: i for i, key in enumerate(st)} for st in self.states]
        self.W = []
        for k in range(L):
            Wk = {}
            for (a, b), M in edges[k].items():
                Wk[(index[k][a], index[k + 1][b])] = np.asarray(M, dtype=np.float64)
            self.W.append(Wk)
        self.dq = [np.array([_state_dq(key) for key in st], dtype=np.int64).reshape(-1, 2)
                   for st in self.states]
        self.index = index

    def bond_dim(self, c):
        return len(self.states[c])

    def sparse_site(self, k):
        """W[k] as 16 sparse (n_k x n_{k+1}) matrices, one per (s_out, s_in)."""
        n0, n1 = len(self.states[k]), len(self.states[k + 1])
        out = {}
        for s in range(4):
            for t in range(4):
                r, c, v = [], [], []
                for (i, j), M in self.W[k].items():
                    if M[s, t] != 0.0:
                        r.append(i)
                        c.append(j)
                        v.append(M[s, t])
                out[(s, t)] = sp.csr_matrix((v, (r, c)), shape=(n0, n1))
        return out


def _state_dq(key):
    if key[0] in ("I", "F"):
        return (0, 0)
    n = t = 0
    for (_, s, d) in key[1]:
        c = _charge(s, d)
        n += c[0]
        t += c[1]
    if key[0] == "P":
        return (n, t)
    return (-n, -t)


def _sort_key(key):
    order = {"I": 0, "P": 1, "S": 2, "F": 3}
    return (order[key[0]], key[1] if len(key) > 1 else ())


def mpo_to_dense(mpo):
    """Contract W[0] ... W[L-1] into the dense 4^L x 4^L matrix (small L only)."""
    L = mpo.L
    m = L // 2
    left = {0: np.ones((1, 1))}
    for k in range(m):
        new = {}
        for (i, j), M in mpo.W[k].items():
            if i in left:
                new[j] = new.get(j, 0.0) + np.kron(left[i], M)
        left = new
    right = {0: np.ones((1, 1))}
    for k in range(L - 1, m - 1, -1):
        new = {}
        for (i, j), M in mpo.W[k].items():
            if j in right:
                new[i] = new.get(i, 0.0) + np.kron(M, right[j])
        right = new
    dim = 4 ** L
    H = np.zeros((dim, dim))
    for w in left:
        if w in right:
            H += np.kron(left[w], right[w])
    return H
