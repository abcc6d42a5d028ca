"""CPU FP64 oracle for the BTA hot path of the spatio-temporal INLA objective.

TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library and its
Python binding) imports, calls or links this package; only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may use it.  It shares no code with the CUDA path: the
only common module is ``synth`` (seeded geometry and random inputs).

Modules
  fem    -- P1 finite elements on the triangle mesh: lumped mass C, stiffness
            G, barycentric interpolation rows (Section II-A.1).
  model  -- theta map, SPDE/AR(1)/Kronecker prior precision, coregional mixing
            (Eq. 11), permutation to BTA order (Section IV-B.1), observation
            operator and Q_c = Q_p + A^T D A (Eq. 4).
  dense  -- "tier D": the plain definitions (dense Cholesky, log-determinant,
            solve, inverse) and extraction of BTA blocks.
  bta    -- "tier B": the block recurrences of the BTA factorisation, solve
            and selected inversion (Section III-A), for sizes where a dense
            N x N matrix does not fit in seconds.  Pinned against tier D.
  fobj   -- the objective f_obj(theta) of Eq. 8 term by term, the central
            finite-difference gradient of Eq. 10, and the adjoint gradient
            (dense or block tier).
  laplace -- f_obj for a non-Gaussian (Poisson) likelihood: Newton
            iterations for the mode x* of the latent field and the Laplace
            approximation at x* (Section II-A.3, Eqs. 4, 7, 8).

Parity status: every function is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` (closed forms, invariants, brute force and
library special cases); none is "parity unpinned".
"""
