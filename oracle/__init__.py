"""FP64 CPU oracle for the D²IP fitting iteration -- TEST INFRASTRUCTURE ONLY.

Plain, slow NumPy restatements of what the paper's method computes, used to check the
CUDA path.  Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the library itself never does, and this package imports
nothing from the library (it shares no code, tables or helpers with the CUDA path).

Modules:
  network -- the residual 3D U-Net phi(theta | Z) (Eq. 2) and its exact backward pass.
  dip     -- the data term of Eq. 4 with the l2 norm, its gradient through J^T, Adam,
             the per-frame fit, UPWS (Eqs. 5-7), TPP (Eqs. 8-9) and ERR.
  tv4d    -- the 4D-TV regulariser (Eqs. 10-13) and its gradient.
  fastres -- the paper-form 3D-FastResUNet (Sec. III-D) as a flagged variant: PyTorch CPU
             float64 forward, gradient by reverse-mode differentiation.

Each function cites the passage it follows.  Pins (brute-force loops, closed forms,
finite differences, library special cases) live in tests/test_oracle_*.py.
"""
