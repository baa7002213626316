"""Writes l30_slice.npz: the oracle's H_eff psi at L=30 on a 3-sector slice.

L=30 orbitals, N=30 electrons, 2S_z=0 (the integrals of the L=30 workload,
seed 1002), a random MPS with D=256 (seed 1003; sites 0..13 left-isometric,
14..29 right-isometric), two-site position b=14 (the mid-chain cut).  The
input vector is the seeded random two-site vector (seed 1004) kept only on
the three largest psi sectors (Sec. II.B step 2, the "3-sector slice");
the oracle's product H_eff psi (Eq. 3 restricted to the MPS span, through
its own environments, enlargement and block products) is stored for every
output sector, with the two elementwise error scales the tests use: the
product of absolute values (BF16x3 bound) and the product of 64-block row
maxima (sliced bound).  Only ``oracle`` and ``inputs`` are called.

    python tests/golden/make_l30_slice.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import inputs  # noqa: E402
from oracle import dmrg as R  # noqa: E402
from oracle import hamiltonian as H  # noqa: E402
from oracle import mpo as M  # noqa: E402

L, N, TSZ, D, B = 30, 30, 0, 256, 14
SEED_INT, SEED_MPS, SEED_PSI = 1002, 1003, 1004


def inflate(a, axis):
    """Every entry replaced by the maximum |entry| of its 64-block along axis."""
    a = np.moveaxis(np.abs(a), axis, -1)
    n = a.shape[-1]
    nb = -(-n // 64)
    pad = np.zeros(a.shape[:-1] + (nb * 64 - n,))
    m = np.concatenate([a, pad], axis=-1).reshape(a.shape[:-1] + (nb, 64)).max(axis=-1)
    return np.moveaxis(np.repeat(m, 64, axis=-1)[..., :n], -1, axis)


def main():
    t0 = time.time()
    h, eri = inputs.make_integrals(L, SEED_INT)
    mp = M.MPO(L, H.hamiltonian_terms(h, eri))
    sites, dims = inputs.make_mps(L, N, TSZ, D, SEED_MPS, n_left=B)
    EL = R.build_left_envs(sites, dims, mp, B)[B]
    ER = R.build_right_envs(sites, dims, mp, B + 2, (N, TSZ))[B + 2]
    He = R.Heff(EL, ER, dims, mp, B)
    psi = He.to_enlarged(inputs.make_psi(dims, B, SEED_PSI), None)
    big = sorted(He.sectors, key=lambda Q: -He.shape[Q][0] * He.shape[Q][1])[:3]
    x = He.flatten({Q: psi[Q] for Q in big})
    y = He.matvec(x)
    # elementwise error scales
    pa = He.unflatten(np.abs(x))
    ya = {Q: np.zeros(s) for Q, s in He.shape.items()}
    yi = {Q: np.zeros(s) for Q, s in He.shape.items()}
    px = He.unflatten(x)
    for (Q, Q2), bl, br in He.pairs:
        if Q2 not in big:
            continue
        ya[Q] += np.einsum("cik,clk->il", np.einsum("cij,jk->cik", np.abs(bl), pa[Q2]), np.abs(br))
        X = np.einsum("cij,jk->cik", inflate(bl, 2), inflate(px[Q2], 0))
        yi[Q] += np.einsum("cik,clk->il", inflate(X, 2), inflate(br, 2))
    np.savez_compressed(os.path.join(HERE, "l30_slice.npz"), x=x, y=y, abs_product=He.flatten(ya),
                        inflated_product=He.flatten(yi),
                        sectors=np.array([[Q[0], Q[1], He.shape[Q][0], He.shape[Q][1]] for Q in He.sectors]),
                        slice_sectors=np.array([[Q[0], Q[1]] for Q in big]),
                        params=np.array([L, N, TSZ, D, B, SEED_INT, SEED_MPS, SEED_PSI]))
    print(f"dim {He.dim}, slice {big}, |y|max {np.abs(y).max():.6g}, {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
