"""Plain FP64 CPU oracle for the macro-element HDG method (arXiv 2302.10917).

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.

It is a slow, literal restatement of the paper's discrete problem:

* the weak form of Section 3.1 (Eqs. mixed/pde/transmission) with the LDG-H
  numerical flux, written as the bilinear forms A, B, C, D and the linear
  forms l, m of Eq. (weak_form);
* the macro-element spaces of Section 3.2 (C0 piecewise P_p on a uniform
  m-fold simplicial subdivision of each macro-triangle, C0 piecewise P_p on
  each macro-edge for the trace);
* the block system of Eq. (D), its static condensation Eqs.
  (global_problem)/(local_problem), and the four-step matrix-free apply of
  Section 3.3.2 with the D^-1 preconditioner of Section 6.1;
* GMRES (Section 6.1) and the local back-solve Eq. (local_matrix_problem);
* the counting formulas of Section 5 (Tables 1-2);
* macro-elements of uneven refinement level with faces at the finer side's
  level (Section 4.2, ``levels.py``);
* the face-block preconditioner (the inverted diagonal face blocks of the
  condensed operator, not in the paper; ``precond.py``).

Every element matrix is integrated in PHYSICAL coordinates, sub-triangle by
sub-triangle, with a Gauss rule built here from the Legendre recurrence. It
shares no code, table or helper with the CUDA library.
"""
