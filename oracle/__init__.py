"""FP64 CPU oracle for the HDG linearize + condense hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path (the
CUDA library under ``paper_2608_27863_gb300``) never calls it, and it never calls
the product path: the two share no code, headers, tables or helpers.  Inputs
come from ``synth`` (seeded generators that hold none of the method's
arithmetic).

It is a plain, slow, obviously correct restatement of the paper's equations:

* ``refelem``  -- Gauss / Gauss-Lobatto rules and Lagrange bases (Sec. 2.2 spaces);
* ``mesh``     -- faces, orientation permutations, block-sparse pattern;
* ``physics``  -- convective / viscous / artificial-viscosity fluxes (Sec. 2.1);
* ``hdg``      -- the element residuals R_q, R_u, R_uhat (eq. hdg-weak, the DIRK
  stage residual), their Jacobians by complex-step differentiation, the dense
  static condensation of eqs. newton-local-block / local-elimination /
  schur-trace, assembly, trace matvec and interior recovery.

Every function states the passage it follows.  Pins against what the paper
and the mathematics fix live in ``tests/test_oracle_*.py``.
"""
