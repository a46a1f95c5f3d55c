"""FP64 CPU oracle for the MBL matrix-free eigensolver hot path.

TEST INFRASTRUCTURE ONLY.  Only tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import this package.  It
shares no code with the CUDA library under ``paper_2012_00217_gb300/``.

Modules:
  hamiltonian -- basis, ranks, diagonal, (H - sigma)X and dense builders
                 (Sec. 2.1, Eq. (model), Eq. (Hmatrix)).
  solver      -- Jacobi-preconditioned PCG, folded-spectrum LOBPCG, final
                 Rayleigh-Ritz with H, spectrum bounds (Sec. 3.2, Sec. 6.2).
  closed_form -- Jordan-Wigner free-fermion spectrum at delta = 0 and other
                 closed forms used to pin the above.
  observables -- the adjacent gap ratio of converged eigenvalues and the
                 half-chain entanglement entropy of eigenvectors (Sec. 2.2).
"""
