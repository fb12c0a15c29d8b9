"""Plain FP64 CPU oracle of the prismatic DG ocean-model hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or run
anything in this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` use it.  It shares no code, table or
constant with the CUDA library; both read only the seeded inputs of ``workloads``.

Every function is written from the paper's statement of the method (arXiv
2605.16082): the primitive equations (Eqs. 1-6), the split momentum equations
(Eqs. 7-10), the discrete 3D step (Eqs. 11-14), the matrix-free column systems
(Eqs. 15-17, Algorithm 1), the assembled column solves (Sec. 2.4) and the 3D/2D
transport consistency (Sec. 2.2, Sec. 2.5, Eq. 18).  Where the paper defers to its
supporting information (not available) the oracle follows a stated reading of the
continuous equations, given in each function's docstring.

Style: numpy, vectorised over prisms / triangles, explicit loops over quadrature
points and basis functions, numerical quadrature for every integral (no
closed-form element matrices), dense ``numpy.linalg.solve`` for every column
system.  Slow and obviously correct by design.

Parity status per function is stated in its docstring; functions whose result is
not fixed by anything other than the reading itself say "parity unpinned".
"""
