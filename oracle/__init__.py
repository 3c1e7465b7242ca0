"""CPU oracle for the shadow-QEq Coulomb hot path (TEST INFRASTRUCTURE ONLY).

This package is a plain, slow FP64 restatement of what the paper's method
computes.  It is checked against closed forms and invariants in the CPU test
suite.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  The CUDA library never calls it, and it never calls
the CUDA library.

Modules:
  neighbors  -- position wrap and brute-force neighbour pairs (Alg. 1, exact set)
  ewald      -- real-space sum (Eq. ewald_real + Gaussian correction), explicit
                k-vector sum (Eq. ewald_rec), self term (Eq. ewald_self), smooth
                PME (Alg. 2) and the assembled potential operator v = Phi q
  qeq        -- dense QEq solve (Eq. linear_qeq), shadow charges
                (Eq. diag_linear_qeq), Jacobian action and low-rank Krylov
                kernel (Sec. 3.5), shadow forces and energy, XL-BOMD integrator
  short_range -- analytic flexible-water stand-in for V_short (not from the
                paper; parity unpinned)
"""
