"""Plain FP64 CPU oracle of the real-space FLO-SIC orbital-SIC step.

TEST INFRASTRUCTURE ONLY.  The oracle exists to check the CUDA path; only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA path and never
imports the ``paper_2108_01186_gb300`` package.

``flosic_oracle.c`` holds the grid loops (Laplacian, multipole boundary
values, conjugate-gradient Poisson solve, tricubic interpolation, LSDA);
``flosic.py`` holds the steps of the method in the paper's order (Fermi
orbitals Eqs. 6-8, Loewdin orthogonalisation, PZ-SIC energy Eq. 1, the
averaged SIC potential Eq. 13, and the FOD gradient by reverse mode and by
the Pederson form Eq. 9).
"""
from .flosic import *  # noqa: F401,F403
from .flosic import build_library, lib  # noqa: F401
