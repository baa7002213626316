"""Two-site DMRG on block-sparse U(1)xU(1) tensors (Sec. II.B, Fig. 3a; Eqs. 2-3).

Test infrastructure: plain FP64 numpy, slow on purpose.  Steps, in the order
Sec. II.B lists them for one DMRG iteration at the two-site cut (b, b+1):

1. pre-processing: the environment of the left block (orbitals 0..b-1) and
   of the right block (orbitals b+2..L-1) -- the renormalised operator sets
   of ``mpo`` -- are enlarged by orbital b (left) and orbital b+1 (right):
   O^Lx_c = sum_a W_b[a,c] (x) E^L[a] and O^xR_c = sum_e W_{b+1}[c,e] (x) E^R[e];
2. diagonalisation: H_eff psi = sum_c O^Lx_c psi (O^xR_c)^T (Eq. 3 restricted
   to the span of the MPS, Eq. 2) inside a Davidson solver;
3. post-processing: per-sector reduced density matrix, global descending sort,
   keep at most D states (the new basis of the enlarged block), the
   renormalisation U^T O^Lx U of every operator, and the transformed start
   vector of the next step.

Block-sparse storage: an operator set is a dict
{(q_out, q_in): (state ids, array (n_states, rows, cols))}; a wavefunction in
enlarged form is a dict {Q: array (dim L-block(Q), dim R-block(Q))} where Q
is the quantum number of the enlarged left block (counted from the left).

Readings where the paper is silent: Davidson with diagonal preconditioner,
max subspace 24, restart keeping 4, ||r|| <= 1e-8, at most 200 products; the
truncation keeps at most D states, moves the cut down to the start of a
group of eigenvalues equal to relative 1e-10 when the group straddles the
cut, drops sqrt(lambda) <= 1e-13 sqrt(lambda_max), keeps at least one; a sweep
is left-to-right over cuts 0..L-3 then right-to-left over L-2..1.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

QS = ((0, 0), (1, 1), (1, -1), (2, 0))


def _add(a, b):
    return (a[0] + b[0], a[1] + b[1])


def _sub(a, b):
    return (a[0] - b[0], a[1] - b[1])


# ----------------------------------------------------------------------------
# bases of the enlarged blocks
# ----------------------------------------------------------------------------

def left_enlarged_basis(dims_k):
    """Sectors of (left block at cut k) + orbital k: Q -> [(s, q_prev, off, size)], dim."""
    segs = {}
    for s, qs in enumerate(QS):
        for q, d in dims_k.items():
            segs.setdefault(_add(q, qs), []).append([s, q, 0, d])
    out = {}
    for Q, lst in segs.items():
        lst.sort(key=lambda x: x[0])
        off = 0
        for x in lst:
            x[2] = off
            off += x[3]
        out[Q] = ([tuple(x) for x in lst], off)
    return out


def right_enlarged_basis(dims_k1):
    """Sectors of orbital k + (right block at cut k+1), labelled at cut k."""
    segs = {}
    for s, qs in enumerate(QS):
        for q, d in dims_k1.items():
            segs.setdefault(_sub(q, qs), []).append([s, q, 0, d])
    out = {}
    for Q, lst in segs.items():
        lst.sort(key=lambda x: x[0])
        off = 0
        for x in lst:
            x[2] = off
            off += x[3]
        out[Q] = ([tuple(x) for x in lst], off)
    return out


# ----------------------------------------------------------------------------
# environments
# ----------------------------------------------------------------------------

def left_env_start(mpo):
    return {((0, 0), (0, 0)): (np.array([mpo.index[0][("I",)]]), np.ones((1, 1, 1)))}


def right_env_start(mpo, Qtot):
    return {(Qtot, Qtot): (np.array([mpo.index[mpo.L][("F",)]]), np.ones((1, 1, 1)))}


def _by_dq(dq):
    groups = {}
    for i, d in enumerate(map(tuple, dq)):
        groups.setdefault(d, []).append(i)
    return {d: np.array(v) for d, v in groups.items()}


def enlarge_left(EL, dims_k, mpo, k):
    """O^Lx_c = sum_a W_k[a, c] (x) E^L[a] for the states c of cut k+1."""
    basis = left_enlarged_basis(dims_k)
    Wsp = mpo.sparse_site(k)
    groups = _by_dq(mpo.dq[k + 1])
    out = {}
    for Q2, (seg2, dim2) in basis.items():
        for dq, C in groups.items():
            Q = _add(Q2, dq)
            if Q not in basis:
                continue
            seg, dim = basis[Q]
            blk = np.zeros((len(C), dim, dim2))
            hit = False
            for (s, qp, off, sz) in seg:
                for (t, qp2, off2, sz2) in seg2:
                    if (qp, qp2) not in EL:
                        continue
                    A, data = EL[(qp, qp2)]
                    Wst = Wsp[(s, t)][A][:, C]
                    if Wst.nnz == 0:
                        continue
                    hit = True
                    blk[:, off:off + sz, off2:off2 + sz2] += \
                        (Wst.T @ data.reshape(len(A), -1)).reshape(len(C), sz, sz2)
            if hit:
                mask = np.abs(blk).reshape(len(C), -1).max(axis=1) > 0
                if mask.any():
                    out[(Q, Q2)] = (C[mask], blk[mask])
    return out, basis


def enlarge_right(ER, dims_k1, mpo, k):
    """O^xR_c = sum_e W_k[c, e] (x) E^R[e] for the states c of cut k."""
    basis = right_enlarged_basis(dims_k1)
    Wsp = mpo.sparse_site(k)
    groups = _by_dq(mpo.dq[k])
    out = {}
    for Q2, (seg2, dim2) in basis.items():
        for dq, C in groups.items():
            Q = _add(Q2, dq)
            if Q not in basis:
                continue
            seg, dim = basis[Q]
            blk = np.zeros((len(C), dim, dim2))
            hit = False
            for (s, qn, off, sz) in seg:
                for (t, qn2, off2, sz2) in seg2:
                    if (qn, qn2) not in ER:
                        continue
                    E, data = ER[(qn, qn2)]
                    Wst = Wsp[(s, t)][C][:, E]
                    if Wst.nnz == 0:
                        continue
                    hit = True
                    blk[:, off:off + sz, off2:off2 + sz2] += \
                        (Wst @ data.reshape(len(E), -1)).reshape(len(C), sz, sz2)
            if hit:
                mask = np.abs(blk).reshape(len(C), -1).max(axis=1) > 0
                if mask.any():
                    out[(Q, Q2)] = (C[mask], blk[mask])
    return out, basis


def renormalise(O, U):
    """E_new[(q, q2)] = U_q^T O[(q, q2)] U_q2 for every stored block."""
    out = {}
    for (Q, Q2), (C, blk) in O.items():
        if Q in U and Q2 in U:
            out[(Q, Q2)] = (C, np.einsum("ia,cij,jb->cab", U[Q], blk, U[Q2]))
    return out


def left_isometry_from_site(A, dims_k, dims_k1):
    """U_Q (dim Lx(Q) x dims_k1[Q]) from a left-isometric site tensor."""
    basis = left_enlarged_basis(dims_k)
    U = {}
    for Q, m in dims_k1.items():
        seg, dim = basis[Q]
        u = np.zeros((dim, m))
        for (s, qp, off, sz) in seg:
            if (qp, s) in A:
                u[off:off + sz] = A[(qp, s)]
        U[Q] = u
    return U


def right_isometry_from_site(B, dims_k, dims_k1):
    """V_Q (dim xR(Q) x dims_k[Q]) from a right-isometric site tensor."""
    basis = right_enlarged_basis(dims_k1)
    V = {}
    for Q, m in dims_k.items():
        seg, dim = basis[Q]
        v = np.zeros((dim, m))
        for (s, qn, off, sz) in seg:
            if (Q, s) in B:
                v[off:off + sz] = B[(Q, s)].T
        V[Q] = v
    return V


def build_left_envs(sites, dims, mpo, upto):
    """Left environments at cuts 0..upto from left-isometric sites 0..upto-1."""
    envs = [left_env_start(mpo)]
    for k in range(upto):
        O, _ = enlarge_left(envs[-1], dims[k], mpo, k)
        envs.append(renormalise(O, left_isometry_from_site(sites[k], dims[k], dims[k + 1])))
    return envs


def build_right_envs(sites, dims, mpo, downto, Qtot):
    """Right environments at cuts L..downto from right-isometric sites."""
    L = mpo.L
    envs = {L: right_env_start(mpo, Qtot)}
    for k in range(L - 1, downto - 1, -1):
        O, _ = enlarge_right(envs[k + 1], dims[k + 1], mpo, k)
        envs[k] = renormalise(O, right_isometry_from_site(sites[k], dims[k], dims[k + 1]))
    return envs


# ----------------------------------------------------------------------------
# effective Hamiltonian at the two-site cut
# ----------------------------------------------------------------------------

class Heff:
    """H_eff at sites (b, b+1) built from E^L (cut b) and E^R (cut b+2)."""

    def __init__(self, EL, ER, dims, mpo, b):
        self.OL, self.bL = enlarge_left(EL, dims[b], mpo, b)
        self.OR, self.bR = enlarge_right(ER, dims[b + 2], mpo, b + 1)
        self.sectors = sorted(Q for Q in self.bL if Q in self.bR)
        self.shape = {Q: (self.bL[Q][1], self.bR[Q][1]) for Q in self.sectors}
        self.offsets = {}
        off = 0
        for Q in self.sectors:
            self.offsets[Q] = off
            off += self.shape[Q][0] * self.shape[Q][1]
        self.dim = off
        self.pairs = []
        for key in self.OL:
            if key in self.OR and key[0] in self.shape and key[1] in self.shape:
                CL, bl = self.OL[key]
                CR, br = self.OR[key]
                common, il, ir = np.intersect1d(CL, CR, return_indices=True)
                if len(common):
                    self.pairs.append((key, bl[il], br[ir]))

    def unflatten(self, x):
        return {Q: x[self.offsets[Q]:self.offsets[Q] + a * b].reshape(a, b)
                for Q, (a, b) in self.shape.items()}

    def flatten(self, psi):
        x = np.zeros(self.dim)
        for Q, (a, b) in self.shape.items():
            if Q in psi:
                x[self.offsets[Q]:self.offsets[Q] + a * b] = psi[Q].ravel()
        return x

    def apply(self, psi):
        """Y[Q] = sum_{Q2} sum_c O^Lx_c[Q,Q2] psi[Q2] O^xR_c[Q,Q2]^T."""
        Y = {Q: np.zeros(s) for Q, s in self.shape.items()}
        for (Q, Q2), bl, br in self.pairs:
            X = np.einsum("cij,jk->cik", bl, psi[Q2])
            Y[Q] += np.einsum("cik,clk->il", X, br)
        return Y

    def matvec(self, x):
        return self.flatten(self.apply(self.unflatten(x)))

    def diagonal(self):
        d = {Q: np.zeros(s) for Q, s in self.shape.items()}
        for (Q, Q2), bl, br in self.pairs:
            if Q == Q2:
                d[Q] += np.einsum("ci,cj->ij", np.einsum("cii->ci", bl), np.einsum("cjj->cj", br))
        return self.flatten(d)

    def to_enlarged(self, psi4, b_dims_left):
        """(q, s1, s2) blocks -> {Q: matrix} on the enlarged bases."""
        out = {Q: np.zeros(s) for Q, s in self.shape.items()}
        for (q, s1, s2), blk in psi4.items():
            Q = _add(q, QS[s1])
            segL = {s: (off, sz) for (s, qp, off, sz) in self.bL[Q][0]}
            segR = {s: (off, sz) for (s, qn, off, sz) in self.bR[Q][0]}
            r0, rn = segL[s1]
            c0, cn = segR[s2]
            out[Q][r0:r0 + rn, c0:c0 + cn] = blk
        return out

    def to_blocks(self, psi):
        out = {}
        for Q, M in psi.items():
            for (s1, qp, r0, rn) in self.bL[Q][0]:
                for (s2, qn, c0, cn) in self.bR[Q][0]:
                    out[(qp, s1, s2)] = M[r0:r0 + rn, c0:c0 + cn].copy()
        return out


# ----------------------------------------------------------------------------
# Davidson (Sec. II.A: "Lanczos or Davidson")
# ----------------------------------------------------------------------------

def davidson(matvec, diag, x0, tol=1e-8, max_sub=24, keep=4, max_mv=200):
    """Lowest eigenpair; returns (theta, x, ||r||, matvecs)."""
    x0 = x0 / np.linalg.norm(x0)
    V = [x0]
    AV = [matvec(x0)]
    nmv = 1
    while True:
        Vm = np.array(V)
        AVm = np.array(AV)
        Hs = Vm @ AVm.T
        Hs = 0.5 * (Hs + Hs.T)
        th, S = np.linalg.eigh(Hs)
        x = S[:, 0] @ Vm
        ax = S[:, 0] @ AVm
        r = ax - th[0] * x
        rn = float(np.linalg.norm(r))
        if rn <= tol or nmv >= max_mv:
            return float(th[0]), x / np.linalg.norm(x), rn, nmv
        den = diag - th[0]
        den = np.where(np.abs(den) < 1e-12, np.copysign(1e-12, den), den)
        t = -r / den
        for _ in range(2):
            t = t - Vm.T @ (Vm @ t)
        tn = np.linalg.norm(t)
        if tn < 1e-14:
            t = r - Vm.T @ (Vm @ r)
            tn = np.linalg.norm(t)
        t /= tn
        if len(V) >= max_sub:
            kk = min(keep, len(V))
            V = list(S[:, :kk].T @ Vm)
            AV = list(S[:, :kk].T @ AVm)
            Vm = np.array(V)
            for _ in range(2):
                t = t - Vm.T @ (Vm @ t)
            t /= np.linalg.norm(t)
        V.append(t)
        AV.append(matvec(t))
        nmv += 1


# ----------------------------------------------------------------------------
# truncation (post-processing, Sec. II.B step 3)
# ----------------------------------------------------------------------------

def select_states(evals_by_sector, D, tie_rel=1e-10, zero_rel=1e-13):
    """Global descending selection; returns {Q: number kept}, truncation weight."""
    allv = []
    for Q, ev in evals_by_sector.items():
        for i, v in enumerate(ev):
            allv.append((float(v), Q, i))
    allv.sort(key=lambda x: (-x[0], x[1], x[2]))
    lam = np.array([max(v, 0.0) for v, _, _ in allv])
    sig = np.sqrt(lam)
    n = len(allv)
    keep = min(D, n)
    if keep < n and keep > 0:
        ref = sig[keep - 1]
        if abs(sig[keep] - ref) <= tie_rel * max(ref, 1e-300):
            j = keep - 1
            while j > 0 and abs(sig[j - 1] - ref) <= tie_rel * max(ref, 1e-300):
                j -= 1
            keep = max(j, 1)
    smax = sig[0] if n else 0.0
    while keep > 1 and sig[keep - 1] <= zero_rel * smax:
        keep -= 1
    kept = {}
    for v, Q, i in allv[:keep]:
        kept[Q] = kept.get(Q, 0) + 1
    weight = float(max(0.0, 1.0 - lam[:keep].sum()))
    return kept, weight


def truncate_left(psi, D):
    """rho = psi psi^T per sector; returns (U: {Q: dim x kept}, C = U^T psi, weight)."""
    ev, vec = {}, {}
    for Q, M in psi.items():
        w, v = np.linalg.eigh(M @ M.T)
        ev[Q] = w[::-1]
        vec[Q] = v[:, ::-1]
    kept, weight = select_states(ev, D)
    U = {Q: vec[Q][:, :m] for Q, m in kept.items()}
    C = {Q: U[Q].T @ psi[Q] for Q in U}
    return U, C, weight


def truncate_right(psi, D):
    """rho = psi^T psi per sector; returns (V: {Q: dim x kept}, C = psi V, weight)."""
    ev, vec = {}, {}
    for Q, M in psi.items():
        w, v = np.linalg.eigh(M.T @ M)
        ev[Q] = w[::-1]
        vec[Q] = v[:, ::-1]
    kept, weight = select_states(ev, D)
    V = {Q: vec[Q][:, :m] for Q, m in kept.items()}
    C = {Q: psi[Q] @ V[Q] for Q in V}
    return V, C, weight


# ----------------------------------------------------------------------------
# sweep driver
# ----------------------------------------------------------------------------

class DMRG:
    """Two-site DMRG from a right-isometric MPS (all sites), FP64."""

    def __init__(self, mpo, sites, dims, N, tsz, D, tol=1e-8):
        self.mpo = mpo
        self.L = mpo.L
        self.sites = [dict(s) for s in sites]
        self.dims = [dict(d) for d in dims]
        self.Qtot = (N, tsz)
        self.D = D
        self.tol = tol
        L = self.L
        self.ER = build_right_envs(self.sites, self.dims, mpo, 2, self.Qtot)
        self.EL = {0: left_env_start(mpo)}
        self.b = 0
        # two-site start vector from B_0 B_1
        psi4 = {}
        for (q, s0), B0 in self.sites[0].items():
            q1 = _add(q, QS[s0])
            for s1 in range(4):
                if (q1, s1) in self.sites[1]:
                    psi4[(q, s0, s1)] = B0 @ self.sites[1][(q1, s1)]
        self.psi4 = psi4
        self.log = []

    def optimise(self, b):
        H = Heff(self.EL[b], self.ER[b + 2], self.dims, self.mpo, b)
        x0 = H.flatten(H.to_enlarged(self.psi4, None))
        if np.linalg.norm(x0) < 1e-12:
            x0 = np.random.default_rng(b).normal(size=H.dim)
        e, x, rn, nmv = davidson(H.matvec, H.diagonal(), x0, tol=self.tol)
        return H, e, H.unflatten(x), rn, nmv

    def step_right(self, b):
        H, e, psi, rn, nmv = self.optimise(b)
        U, C, w = truncate_left(psi, self.D)
        self.dims[b + 1] = {Q: u.shape[1] for Q, u in U.items()}
        A = {}
        for Q, u in U.items():
            for (s, qp, off, sz) in H.bL[Q][0]:
                A[(qp, s)] = u[off:off + sz].copy()
        self.sites[b] = A
        self.EL[b + 1] = renormalise(H.OL, U)
        psi4 = {}
        Bn = self.sites[b + 2]
        for Q, c in C.items():
            for (s2, qn, off, sz) in H.bR[Q][0]:
                for s3 in range(4):
                    if (qn, s3) in Bn:
                        psi4[(Q, s2, s3)] = c[:, off:off + sz] @ Bn[(qn, s3)]
        self.psi4 = psi4
        self.log.append(dict(b=b, dir=1, e=e, resid=rn, nmv=nmv, trunc=w))
        return e

    def step_left(self, b):
        H, e, psi, rn, nmv = self.optimise(b)
        V, C, w = truncate_right(psi, self.D)
        self.dims[b + 1] = {Q: v.shape[1] for Q, v in V.items()}
        B = {}
        for Q, v in V.items():
            for (s, qn, off, sz) in H.bR[Q][0]:
                B[(Q, s)] = v[off:off + sz].T.copy()
        self.sites[b + 1] = B
        self.ER[b + 1] = renormalise(H.OR, V)
        psi4 = {}
        Ap = self.sites[b - 1]
        for Q, c in C.items():
            for (s1, qp, off, sz) in H.bL[Q][0]:
                for s0 in range(4):
                    q0 = _sub(qp, QS[s0])
                    if (q0, s0) in Ap:
                        psi4[(q0, s0, s1)] = Ap[(q0, s0)] @ c[off:off + sz]
        self.psi4 = psi4
        self.log.append(dict(b=b, dir=-1, e=e, resid=rn, nmv=nmv, trunc=w))
        return e

    def sweep(self):
        L = self.L
        es = []
        for b in range(0, L - 2):
            es.append(self.step_right(b))
        for b in range(L - 2, 0, -1):
            es.append(self.step_left(b))
        return es[-1], min(es)


# ----------------------------------------------------------------------------
# Fock-space projection P^T H P psi (pin for H_eff psi, L <= 10)
# ----------------------------------------------------------------------------

def left_basis_vectors(sites, dims, b):
    """Columns = left-block states at cut b as vectors in the 4^b space."""
    vec = {(0, 0): np.ones((1, 1))}
    for k in range(b):
        new = {}
        for Q, m in dims[k + 1].items():
            T = np.zeros((4 ** k, 4, m))
            for s, qs in enumerate(QS):
                qp = _sub(Q, qs)
                if (qp, s) in sites[k] and qp in vec:
                    T[:, s, :] += vec[qp] @ sites[k][(qp, s)]
            new[Q] = T.reshape(4 ** (k + 1), m)
        vec = new
    return vec


def right_basis_vectors(sites, dims, b2, L):
    """Rows = right-block states at cut b2 as vectors in the 4^(L-b2) space."""
    Qtot = next(iter(dims[L]))
    vec = {Qtot: np.ones((1, 1))}
    for k in range(L - 1, b2 - 1, -1):
        new = {}
        for Q, m in dims[k].items():
            T = np.zeros((m, 4, 4 ** (L - k - 1)))
            for s, qs in enumerate(QS):
                qn = _add(Q, qs)
                if (Q, s) in sites[k] and qn in vec:
                    T[:, s, :] += sites[k][(Q, s)] @ vec[qn]
            new[Q] = T.reshape(m, 4 ** (L - k))
        vec = new
    return vec


def heff_fock(H_sparse, sites, dims, b, psi4, L):
    """P^T H P psi with P the MPS isometry around sites (b, b+1)."""
    Lv = left_basis_vectors(sites, dims, b)
    Rv = right_basis_vectors(sites, dims, b + 2, L)
    nl, nr = 4 ** b, 4 ** (L - b - 2)
    full = np.zeros((nl, 4, 4, nr))
    for (q, s1, s2), blk in psi4.items():
        qn = _add(_add(q, QS[s1]), QS[s2])
        full[:, s1, s2, :] += Lv[q] @ blk @ Rv[qn]
    Hf = (H_sparse @ full.ravel()).reshape(nl, 4, 4, nr)
    out = {}
    for (q, s1, s2), blk in psi4.items():
        qn = _add(_add(q, QS[s1]), QS[s2])
        out[(q, s1, s2)] = Lv[q].T @ Hf[:, s1, s2, :] @ Rv[qn].T
    return out


def occupation_to_determinant(L, fci):
    """Map of the 4^L occupation basis onto FCI determinants.

    Returns (idx, ia, ib, sign) for the basis states with the FCI's (N, 2S_z):
    the site-ordered product prod_i (a+_{i up})^na_i (a+_{i dn})^nb_i |0> equals
    sign * |Ia Ib> with sign = (-1)^(sum_i nb_i * #{j > i : na_j = 1}).
    """
    ia_of = {s: k for k, s in enumerate(fci.sa)}
    ib_of = {s: k for k, s in enumerate(fci.sb)}
    idx, ia, ib, sg = [], [], [], []
    for x in range(4 ** L):
        occ = [(x // 4 ** (L - 1 - i)) % 4 for i in range(L)]
        na = [1 if o in (1, 3) else 0 for o in occ]
        nb = [1 if o in (2, 3) else 0 for o in occ]
        a = sum(1 << i for i in range(L) if na[i])
        b = sum(1 << i for i in range(L) if nb[i])
        if a in ia_of and b in ib_of:
            par = sum(nb[i] * sum(na[i + 1:]) for i in range(L)) % 2
            idx.append(x)
            ia.append(ia_of[a])
            ib.append(ib_of[b])
            sg.append(-1.0 if par else 1.0)
    return np.array(idx), np.array(ia), np.array(ib), np.array(sg)


def heff_fock_fci(fci, sites, dims, b, psi4, L, occmap=None):
    """P^T H P psi with H applied as the full-CI sigma vector (Knowles-Handy)."""
    if occmap is None:
        occmap = occupation_to_determinant(L, fci)
    idx, ia, ib, sg = occmap

    class _Sigma:
        shape = (4 ** L, 4 ** L)

        def __matmul__(self, v):
            C = np.zeros(fci.shape)
            C[ia, ib] = sg * v[idx]
            S = fci.sigma(C)
            out = np.zeros(4 ** L)
            out[idx] = sg * S[ia, ib]
            return out

    return heff_fock(_Sigma(), sites, dims, b, psi4, L)
