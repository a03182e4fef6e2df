"""CPU FP64 oracle for the time-stepper stability method (Loiseau et al.,
"Time-stepping and Krylov methods for large-scale instability problems").

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain, obviously-correct
reference that the CUDA path is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  The product library never calls it, and
it shares no code with ``paper_1804_03859_gb300`` (the only shared module is
the seeded input generator ``paper_1804_03859_gb300.inputs``, which holds none
of the method's arithmetic).

Modules
-------
ns2d    : the 2D vorticity-streamfunction time-stepper (nonlinear and
          linearised), i.e. the black-box propagator of Sec. 3 (Eqs. 28-30,
          x -> exp(TA) x) and the nonlinear map G of Eq. 2 / Eq. 41.
krylov  : Algorithm 1 (m-step Arnoldi, Sec. 3.2.1) with a second classical
          Gram-Schmidt pass, Ritz pairs and the residual estimate of Eq. 63,
          and the Krylov-Schur restart of Sec. 3.2.2.
sfd     : selective frequency damping, Eq. 40 (Sec. 3.1.1).
dense   : explicit assembly of M = exp(TA) and of the semi-discrete A by
          columns (only feasible on small grids), used to pin the above.

Every function is FP64 numpy; numpy.fft and numpy/scipy dense linear algebra
serve as library steps.  Functions whose correctness has no independent pin
say "parity unpinned" in their docstring.
"""
