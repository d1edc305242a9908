"""GB300-native quasi-orthogonal inverse-operator eigensolver (Wang & Zhou,
arXiv 2605.25149): C-ABI library ``libhq`` with hand-written sm_103a kernels
and a thin ctypes binding (``paper_2605_25149_gb300.hq``).

Importing the package does not load the CUDA library; ``hq`` does, and fails
loudly if it has not been built.
"""
