"""Plain, slow FP64 CPU oracle for the two-site DMRG hot path (test infrastructure).

This package is test infrastructure.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  The CUDA library never calls it and
shares no code with it; the two meet only through the seeded generators in
``inputs``.

What it computes, and from which passage of arXiv:2412.04676:

* ``hamiltonian``  Eq. 1 with spin labels (chemist (ij|kl) integrals, the 1/2
  of the two-body sum, spin-conserving terms); a dense Jordan-Wigner matrix
  for L <= 6 and a determinant-string full-CI sigma vector (Knowles-Handy) with
  a Lanczos solver -- the pins for everything below.
* ``mpo``          Eq. 1 written as a sum over terms split at every cut of the
  chain into a left part and a right part (normal operators on the left,
  complementary sums on the right), i.e. the operator sets the environments
  of Sec. II.B carry.
* ``dmrg``         the two-site superblock of Sec. II.B / Fig. 3a:
  environments (pre-processing, step 1), the effective-Hamiltonian product
  H_eff psi of the diagonalisation step (step 2, Eq. 3 restricted to the
  span of the MPS of Eq. 2), Davidson, reduced-density-matrix truncation and
  renormalisation (step 3) and the sweep; plus the Fock-space projection
  P^T H P psi that pins H_eff psi.
* ``pack``         the serialisation of Sec. III.B.2-3: exact size prediction,
  self-contained packages located by their own metadata, byte-exact
  round trip.

Parity unpinned: nothing.  Every function is pinned by a test in
``tests/test_oracle_*.py`` (closed forms, brute force, full CI).
"""
