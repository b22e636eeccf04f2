"""CPU oracle (plain FP64 numpy) for the Wilson-clover operator, its clover term, the
even-odd Schur complement and the even-odd CG solve (``qxd_oracle``), for the Schwarz
alternating procedure with flexible GCR around it (``sap_oracle``), for inexact deflation
with a block-local subspace (``dfl_oracle``) and for three-level multigrid on top of it
(``mg_oracle``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py``.  It shares no code with the CUDA path.  Every function that
has no independent pin says "parity unpinned" in its docstring.
"""
from . import qxd_oracle  # noqa: F401
from . import sap_oracle  # noqa: F401
from . import dfl_oracle  # noqa: F401
from . import mg_oracle  # noqa: F401
