"""FP64 CPU oracle for curvature-regularised confocal NLOS reconstruction.

This package is TEST INFRASTRUCTURE. It is a plain, slow, NumPy float64
restatement of what the GPU library computes, written from the paper
(Sec. 2 forward model, Eq. 2-3; Sec. 3 object-domain model, Eq. 4-12 and
Algorithm 1; Sec. 4 dual-domain model, Eq. 13 and Algorithm 2).  It shares no
code, tables or constants with the CUDA path and never imports it.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  The product path
(``paper_2301_00406_gb300``) must never route through it.

Modules
-------
lct     the discrete light-cone-transform operator A = R_t^{-1} H R_z (Eq. 3),
        its transpose, the sampling operator D, a brute-force convolution,
        the physical direct summation of Eq. 2 and the power iteration for
        ||A_D||_2^2.
admm    finite differences, curvature, shrinkage (Eq. 7), the FFT solve
        (Eq. 11), Algorithm 1 and Algorithm 2.
nonconfocal  the midpoint conversion of non-confocal transients into
        confocal ones (Sec. 4, evaluation on non-confocal data).

Parity status of every function is stated in its docstring; all functions
are pinned by ``tests/test_oracle_*.py`` except where the docstring says
"parity unpinned".
"""

from . import lct, admm, nonconfocal  # noqa: F401
