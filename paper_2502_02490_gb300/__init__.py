"""GB300-native O(a)-improved QCD+QED Wilson-clover Dirac operator and solvers.

The compute path is the C-ABI library ``libqxd.so`` (hand-written sm_103a CUDA) behind the
thin ctypes binding in :mod:`paper_2502_02490_gb300.qxd`.  Importing this package loads
nothing; ``from paper_2502_02490_gb300 import qxd`` loads the library and raises if it is
missing.  :mod:`paper_2502_02490_gb300.synth` holds the seeded input generators.
"""
__all__ = ["qxd", "synth"]
