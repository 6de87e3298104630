"""CPU FP64 oracle for the Wilson-Dirac operator and conjugate gradient (arXiv 2111.14958).

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports this package: only ``tests/``,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``
may use it. It shares no code, tables or constants with the CUDA library.

Contents (each function cites the passage of the paper it follows):

* :mod:`oracle.gamma`     -- chiral Euclidean gamma matrices and the spin projectors of Eq. (1).
* :mod:`oracle.wilson`    -- the Wilson-Dirac operator D of Eq. (1) three ways: a vectorised
  stencil (R1), a literal per-site loop (R1'), the paper's coordinate-format (COO) matrix with
  its sparse matrix-vector product (R2, Sec. 2), and a dense matrix (R3).
* :mod:`oracle.cg`        -- CG on the normal equations in CGLS form, and the paper's CG on DD^dagger
  (Sec. 2 algorithm) with the squared-norm reading.
* :mod:`oracle.freefield` -- closed forms for unit links: the momentum-space symbol D(p), the
  eigenvalues of D^dagger D, and an FFT solver.

Parity status: every function is pinned by a ``-m "not gpu"`` test against a closed form, brute
force or an invariant (see ``tests/test_oracle_*.py``); none is "parity unpinned".
"""
from . import gamma, wilson, cg, freefield  # noqa: F401
