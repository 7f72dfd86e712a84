"""CPU oracle for the hierarchical recursive precision Cholesky (HRP).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or link
anything under ``oracle/``; only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA path (paper_2601_08082_gb300/): every definition here is
written again from the paper, in plain float64 numpy (float32 / float16 / E4M3
only where the method itself fixes that precision).

Modules
  dense    plain Cholesky, triangular solves, POTRS and error measures
           (the exact definitions the FP64 path must reproduce).
  lowprec  rounding to FP32 / FP16 / FP8-E4M3 and the per-block scaling rule
           of Sec. 3.4.
  tree     the precision-tree descriptor and an emulator that walks Algorithms
           1-3 step by step with the tree's precisions (the definition the
           mixed-precision GPU path is compared against).
  solve    iterative refinement driver (FP64 residual) on top of the above.

Pins: see tests/test_oracle_*.py.  A function whose result is not pinned to
anything outside itself says "parity unpinned" in its docstring.
"""
