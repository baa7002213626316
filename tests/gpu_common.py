"""Shared set-up of the GPU parity tests: the same seeded inputs go to the
library (through the C-ABI) and to the oracle."""
import numpy as np

import inputs
import paper_2412_04676_gb300 as g
from oracle import dmrg as R
from oracle import hamiltonian as H
from oracle import mpo as M


def build_lib():
    from paper_2412_04676_gb300 import build
    build.build()


def heff_case(L, N, tsz, D, seed, b, oracle=True, **kw):
    """GPU context and (optionally) oracle H_eff at two-site position b."""
    h, eri = inputs.make_integrals(L, seed)
    sites, dims = inputs.make_mps(L, N, tsz, D, seed + 1, n_left=b)
    psi4 = inputs.make_psi(dims, b, seed + 2)
    ctx = g.Context(L, N, tsz, D=D, **kw)
    ctx.load_integrals(h, eri)
    ctx.import_mps(sites, [0] * b + [1] * (L - b))
    ctx.build_envs(b)
    He = None
    if oracle:
        mp = M.MPO(L, H.hamiltonian_terms(h, eri))
        EL = R.build_left_envs(sites, dims, mp, b)[b]
        ER = R.build_right_envs(sites, dims, mp, b + 2, (N, tsz))[b + 2]
        He = R.Heff(EL, ER, dims, mp, b)
    return dict(h=h, eri=eri, sites=sites, dims=dims, psi4=psi4, ctx=ctx, He=He)
