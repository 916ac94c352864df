"""Plain, slow, FP64 CPU oracle for the adaptive-multigrid Wilson-Dirac solve.

This package is TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import,
call or execute it.  The product library (``paper_0811_4331_gb300``) never
imports it and shares no code with it: the two meet only through the seeded
input generators in ``paper_0811_4331_gb300/inputs.py``, which hold none of the
method's arithmetic.

Everything here is written from the paper (Clark et al., "The removal of
critical slowing down", Lattice 2008) in numpy complex128, in the paper's order
and notation, without blocking, fusion or reordering:

* ``dirac``     -- the Wilson-Dirac operator D = Dslash + m (Sec. 1, Eq. 1.1 and the text after it)
                   and its 9-point stencil form.
* ``multigrid`` -- MR relaxation (Sec. 3), null-vector relaxation (Sec. 2,
                   adaptive steps 1-3), blockwise QR into P (Sec. 2, Eq. 2.3),
                   R = P^dagger with [gamma5, P] = 0 (Sec. 3, Eq. 3.2),
                   A_c = P^dagger A P (Sec. 2), the alpha-damped coarse-grid
                   correction (Sec. 3, Eq. 3.5), the modified V(2,2) cycle and
                   flexible GCR(50) (Sec. 5).

Pins (tests/test_oracle_*.py, run with ``-m "not gpu"``) check each function
against facts fixed by the paper or by mathematics, never against itself.
"""
