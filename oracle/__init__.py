"""FP64 CPU oracle of the monodomain P1-FEM time step.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or call this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use it.
It shares no code with the CUDA path; its only common dependency is the seeded input
generator ``paper_2510_12011_b300.inputs`` (mesh geometry and parameter sets, no arithmetic
of the method).

What it computes, and where the paper defines it (TorchCor, arXiv 2510.12011):
  * fem.py        P1 tetrahedral mass and stiffness matrices, A = chi*Cm*M + theta*dt*K
                  (Section 2.2, Eq. 2 and the definitions of A and b after Eq. 3)
  * pcg.py        Jacobi-preconditioned conjugate gradients (Section 2.2, Algorithm 1)
  * ionic.py      Mitchell-Schaeffer ionic model with a Rush-Larsen gate (the model is not
                  written out in the paper; our mV mapping is stated in ionic.py)
  * tp06.py       ten Tusscher-Panfilov 2006 (named in Section 2.2, not printed; restated from
                  the model's own publication; pinned by its charge balance and AP features)
  * monodomain.py the operator-split time step (Eq. 2, Eq. 3), stimulus (Section 2.1),
                  extrapolated initial guess (end of Section 2.2) and activation times
                  (Section 2.1, "LAT")
  * mms.py        the manufactured-solution verification (Section 3.1.1, Eqs. 4-8) and a 3D
                  zero-flux variant of it on tetrahedra
  * mlp.py        the learned surrogate's network (forward, loss, gradients) and the exact
                  single-cell window it is trained on
  * partitioned.py Algorithm 1 over row-partitioned host ranks (the multi-GPU design check)

Everything is float64.  Loops are vectorised over elements or nodes with numpy; no blocking,
fusion or reordering beyond the definitions is done.  Pins: see tests/test_oracle_*.py.
"""
