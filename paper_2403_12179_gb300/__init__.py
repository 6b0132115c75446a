"""GB300-native cell-centered geometric multigrid Poisson solver (sm_103a).

The compute path lives in the C-ABI library ``libgbmg.so`` built from ``csrc/``; the Python
module ``paper_2403_12179_gb300.mg`` is a thin ctypes binding over it.  Importing this package
loads nothing: the library is loaded on first use of ``mg`` and raises if it is missing.
"""
