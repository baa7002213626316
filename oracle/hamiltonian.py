"""Eq. 1 of arXiv:2412.04676 (Sec. II.A) with spin labels, and its exact solutions.

Reading of Eq. 1 (the paper leaves the normalisation open): with spatial
orbitals i, j, k, l and spins s, t in {up, dn},

    H = sum_{ij,s} h_ij a+_{is} a_{js}
        + 1/2 sum_{ijkl,s,t} (ij|kl) a+_{is} a+_{kt} a_{lt} a_{js},

chemist-notation (ij|kl), no core energy.  Everything here is FP64.

Local basis of one orbital: 0=|0>, 1=|up>, 2=|dn>, 3=|updn>=c+_up c+_dn|0>.
Jordan-Wigner: a_{is} = P x ... x P (sites < i) x c_s x 1 x ... with
P = diag(1,-1,-1,1) and orbital 0 the leftmost Kronecker factor.
"""
from __future__ import annotations

from itertools import combinations

import numpy as np
import scipy.sparse as sp

UP, DN = 0, 1


def local_ops():
    """Return (c+_up, c+_dn, P) as 4x4 arrays in the local basis above."""
    cu = np.zeros((4, 4))
    cu[1, 0] = 1.0   # |0>  -> |up>
    cu[3, 2] = 1.0   # |dn> -> c+_up c+_dn |0> = |updn>
    cd = np.zeros((4, 4))
    cd[2, 0] = 1.0   # |0>  -> |dn>
    cd[3, 1] = -1.0  # |up> -> c+_dn c+_up |0> = -|updn>
    P = np.diag([1.0, -1.0, -1.0, 1.0])
    return cu, cd, P


def hamiltonian_terms(h, eri, tol: float = 0.0):
    """Eq. 1 as a list of (coefficient, ops) with ops ((orbital, spin, dagger), ...).

    The operator product is read left to right as written in Eq. 1.  Terms
    with a repeated creation or annihilation index vanish and are omitted.
    """
    L = h.shape[0]
    terms = []
    for i in range(L):
        for j in range(L):
            if abs(h[i, j]) > tol:
                for s in (UP, DN):
                    terms.append((float(h[i, j]), ((i, s, 1), (j, s, 0))))
    for i in range(L):
        for j in range(L):
            for k in range(L):
                for l in range(L):
                    v = 0.5 * eri[i, j, k, l]
                    if abs(v) <= tol:
                        continue
                    for s in (UP, DN):
                        for t in (UP, DN):
                            if (i, s) == (k, t) or (l, t) == (j, s):
                                continue
                            terms.append((float(v), ((i, s, 1), (k, t, 1), (l, t, 0), (j, s, 0))))
    return terms


# ----------------------------------------------------------------------------
# Pin (i): dense Jordan-Wigner Hamiltonian from Kronecker products (L <= 6)
# ----------------------------------------------------------------------------

def jw_annihilators(L: int):
    """Sparse 4^L x 4^L annihilators a[i][s] built from Kronecker products."""
    cu, cd, P = local_ops()
    I4 = sp.identity(4, format="csr")
    Ps = sp.csr_matrix(P)
    loc = [sp.csr_matrix(cu.T), sp.csr_matrix(cd.T)]
    a = []
    for i in range(L):
        row = []
        for s in (UP, DN):
            m = sp.identity(1, format="csr")
            for k in range(L):
                f = Ps if k < i else (loc[s] if k == i else I4)
                m = sp.kron(m, f, format="csr")
            row.append(m)
        a.append(row)
    return a


def jw_hamiltonian(h, eri):
    """Eq. 1 as a sparse 4^L x 4^L matrix, term by term from JW operators."""
    L = h.shape[0]
    a = jw_annihilators(L)
    ad = [[x.T.tocsr() for x in row] for row in a]
    dim = 4 ** L
    H = sp.csr_matrix((dim, dim))
    for i in range(L):
        for j in range(L):
            for s in (UP, DN):
                H = H + h[i, j] * (ad[i][s] @ a[j][s])
    for i in range(L):
        for j in range(L):
            for k in range(L):
                for l in range(L):
                    v = 0.5 * eri[i, j, k, l]
                    if v == 0.0:
                        continue
                    for s in (UP, DN):
                        for t in (UP, DN):
                            H = H + v * (ad[i][s] @ ad[k][t] @ a[l][t] @ a[j][s])
    return H.tocsr()


def occupation_labels(L: int):
    """(n, tsz) of every 4^L basis state, orbital 0 most significant."""
    n_loc = np.array([0, 1, 1, 2])
    t_loc = np.array([0, 1, -1, 0])
    n = np.zeros(1, dtype=np.int64)
    t = np.zeros(1, dtype=np.int64)
    for _ in range(L):
        n = (n[:, None] + n_loc[None, :]).ravel()
        t = (t[:, None] + t_loc[None, :]).ravel()
    return n, t


def jw_ground_energy(h, eri, N: int, tsz: int):
    """Lowest eigenvalue of the JW Hamiltonian in the (N, 2S_z) block (numpy eigh)."""
    H = jw_hamiltonian(h, eri)
    n, t = occupation_labels(h.shape[0])
    idx = np.where((n == N) & (t == tsz))[0]
    Hb = H[idx][:, idx].toarray()
    return float(np.linalg.eigvalsh(Hb)[0])


# ----------------------------------------------------------------------------
# Full CI on alpha/beta strings (Knowles-Handy sigma) + Lanczos
# ----------------------------------------------------------------------------

def strings(L: int, n: int):
    """Occupation bit strings with n of L orbitals occupied, lexical order."""
    out = []
    for occ in combinations(range(L), n):
        m = 0
        for o in occ:
            m |= 1 << o
        out.append(m)
    return out


def _popcount(x: int) -> int:
    return bin(x).count("1")


def excitation_operators(L: int, strs):
    """E[i][j] = a+_i a_j on one spin's strings as sparse matrices (with signs)."""
    index = {s: k for k, s in enumerate(strs)}
    dim = len(strs)
    E = [[None] * L for _ in range(L)]
    for i in range(L):
        for j in range(L):
            rows, cols, vals = [], [], []
            for k, I in enumerate(strs):
                if not (I >> j) & 1:
                    continue
                sgn = (-1) ** _popcount(I & ((1 << j) - 1))
                J = I ^ (1 << j)
                if (J >> i) & 1:
                    continue
                sgn *= (-1) ** _popcount(J & ((1 << i) - 1))
                J |= 1 << i
                rows.append(index[J])
                cols.append(k)
                vals.append(float(sgn))
            E[i][j] = sp.csr_matrix((vals, (rows, cols)), shape=(dim, dim))
    return E


class FCI:
    """Determinant full CI in the (N, 2S_z) space; C is an (n_alpha_str, n_beta_str) array.

    Determinant |Ia Ib> = (prod_{i in Ia} a+_{i up})(prod_{i in Ib} a+_{i dn})|0>
    with ascending orbital order inside each product.
    """

    def __init__(self, h, eri, N: int, tsz: int):
        self.h = np.asarray(h, dtype=np.float64)
        self.eri = np.asarray(eri, dtype=np.float64)
        self.L = h.shape[0]
        self.na = (N + tsz) // 2
        self.nb = (N - tsz) // 2
        self.sa = strings(self.L, self.na)
        self.sb = strings(self.L, self.nb)
        self.Ea = excitation_operators(self.L, self.sa)
        self.Eb = excitation_operators(self.L, self.sb)
        # k_ij = h_ij - 1/2 sum_k (ik|kj): the one-body part left after writing
        # the two-body sum as 1/2 sum (ij|kl) E_ij E_kl
        self.k = self.h - 0.5 * np.einsum("ikkj->ij", self.eri)
        self.shape = (len(self.sa), len(self.sb))

    def _E(self, i, j, C):
        return self.Ea[i][j] @ C + (self.Eb[i][j] @ C.T).T

    def sigma(self, C):
        L = self.L
        D = np.empty((L, L) + C.shape)
        for k in range(L):
            for l in range(L):
                D[k, l] = self._E(k, l, C)
        s = np.einsum("ij,ijab->ab", self.k, D)
        G = np.einsum("ijkl,klab->ijab", self.eri, D)
        for i in range(L):
            for j in range(L):
                s += 0.5 * self._E(i, j, G[i, j])
        return s

    def matvec(self, x):
        return self.sigma(x.reshape(self.shape)).ravel()


def lanczos_lowest(matvec, dim: int, seed: int = 0, tol: float = 1e-12, maxiter: int = 300):
    """Lowest eigenpair by Lanczos with full reorthogonalisation."""
    rng = np.random.default_rng(seed)
    v = rng.normal(size=dim)
    v /= np.linalg.norm(v)
    V = [v]
    alpha, beta = [], []
    theta_old = None
    for it in range(min(maxiter, dim)):
        w = matvec(V[-1])
        a = float(V[-1] @ w)
        alpha.append(a)
        w = w - a * V[-1] - (beta[-1] * V[-2] if beta else 0.0)
        Vm = np.array(V)
        for _ in range(2):
            w = w - Vm.T @ (Vm @ w)
        b = float(np.linalg.norm(w))
        T = np.diag(alpha) + np.diag(beta, 1) + np.diag(beta, -1)
        ev, evec = np.linalg.eigh(T)
        theta = ev[0]
        resid = b * abs(evec[-1, 0])
        if resid < tol or b < 1e-14 or (theta_old is not None and abs(theta - theta_old) < tol * 1e-2 and resid < 1e-8):
            break
        theta_old = theta
        beta.append(b)
        V.append(w / b)
    x = np.array(V[: len(alpha)]).T @ evec[:, 0]
    return float(theta), x / np.linalg.norm(x)


def fci_ground_energy(h, eri, N: int, tsz: int):
    f = FCI(h, eri, N, tsz)
    e, _ = lanczos_lowest(f.matvec, f.shape[0] * f.shape[1])
    return e
