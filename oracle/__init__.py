"""CPU oracle for negacyclic polynomial multiplication (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use this package.  It is independent of the CUDA library:
``schoolbook`` is arbitrary-precision Python, ``schoolbook.c`` (driven by
``native``) is a plain C schoolbook with a 192-bit accumulator.
"""
