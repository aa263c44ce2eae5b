"""GB300-native exact negacyclic polynomial multiplication in Z_q[x]/(x^n+1).

The compute path is the C-ABI library ``libpolymul.so`` (hand-written CUDA
for sm_103a, declared in ``include/polymul.h``); ``polymul`` is its thin
ctypes binding and ``workloads`` draws seeded synthetic inputs.  Importing
the package loads nothing: ``from paper_2307_06554_gb300 import polymul``
loads the library and fails loudly if it has not been built.
"""
