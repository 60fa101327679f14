"""CPU oracle for the NCL augmented-Lagrangian / interior-point Newton step.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 restatement of
what the method of "An Augmented Lagrangian Method on GPU for
Security-Constrained AC Optimal Power Flow" (Pacaud et al.) computes, written
so that a reader can check it against the paper by eye.  Only the test suite,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  The CUDA library never calls it and
shares no code with it.

Modules
  scopf_model  polar AC-SCOPF with complementarity (Sections II-III)
  ncl          NCL outer loop (Section IV-A, eq. nclsubpb) and the
               interior-point inner loop with the reduced Newton system
               (Section IV-B, eq. newtonsystem)
  linsolve     dense and simple sparse LDL^T (pivot-free) with inertia
  symbolic     fill-reducing ordering / elimination tree / supernodes
  toys         small MPCCs and NLPs with closed-form answers
  adjoint      sensitivity of the converged solution

Parity status of each function is stated in its docstring; every function is
pinned by a test under tests/ that does not re-derive the same formula.
"""
