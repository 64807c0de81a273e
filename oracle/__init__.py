"""Oracle for the stochastic heat / species diffusion hot path.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its ``cpu_baseline`` leg and ``--impl reference`` arm) may import
this package.  It shares no code with ``paper_2406_12157_gb300``.

* :mod:`oracle.she` -- ctypes binding of the plain FP64 C program
  ``she_oracle.c`` (Philox-4x32-10 + Box-Muller noise, forward-Euler step,
  sampling), Sec. 3 of Garcia et al. (2024).
* :mod:`oracle.theory` -- closed forms and the exact moment recursion of the
  discrete scheme, used to pin the C program to something other than itself.
"""
