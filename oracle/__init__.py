"""CPU FP64 oracle for multi-area WLS state estimation.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU baseline leg
of ``bench.py`` use it.  It shares no code with the CUDA library.

* :mod:`oracle.wls`  - measurement model, analytic Jacobian, centralised
  Gauss-Newton (Sec. 2.1, Eqs. meas_model / wls / gn_normal) and the
  multi-area Schur-condensed Gauss-Newton step (Sec. 3, Eqs. Ek_select,
  block_normal, backsub, local_schur_system, schur_defs, global_assembly).
* :mod:`oracle.mlp`  - FP64 forward/backward of the per-area warm-start MLP
  and its AdamW update (not in the paper; checks the learned warm start).

Parity status: every function is pinned by ``tests/test_oracle_*.py``
against closed forms, independent formulations, finite differences, library
routines or brute force, except where a docstring says "parity unpinned".
"""
