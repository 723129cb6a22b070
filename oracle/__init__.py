"""Plain FP64 CPU oracle for the splitting conic solver (test infrastructure).

This package is the checker, not the product.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py`` (its CPU-baseline leg and its
``--impl reference`` arm) may import it.  It shares no code with the CUDA path
in ``paper_1312_3039_gb300/``; the only common module is the seeded input
generator ``paper_1312_3039_gb300.synth``, which holds none of the method's
arithmetic.

Every function follows a passage of O'Donoghue, Chu, Parikh and Boyd,
"Conic Optimization via Operator Splitting and Homogeneous Self-Dual
Embedding" (cited by section / equation), written for a reader to check by
eye: no blocking, fusion or reordering beyond what the passage states.

Modules:
  cones    -- projections onto the zero, nonnegative, second-order, PSD and
              exponential cones and their duals; membership tests.
  scaling  -- the data equilibration of Sec. 5.
  admm     -- the ADMM iteration on the homogeneous self-dual embedding
              (Eq. "e-SCS" with over-relaxation, Sec. 3.2-3.5), with the
              direct (cached factorisation) and indirect (CG) subspace solves
              of Sec. 4.1, termination and certificates.
  naive    -- the un-simplified ADMM of Eq. "e-SCS-naive" (Sec. 3.1), used
              only to check the simplified iteration against it.
"""
