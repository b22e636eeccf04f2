"""CPU oracle (plain FP64 numpy) for the Wilson-clover operator, its clover term, the
even-odd Schur complement and the even-odd CG solve.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py``.  It shares no code with the CUDA path.  Every function that
has no independent pin says "parity unpinned" in its docstring.
"""
from . import qxd_oracle  # noqa: F401
