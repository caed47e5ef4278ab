"""ORACLE -- test infrastructure only.

A plain, slow, obviously correct FP64 CPU implementation of the paper's
method (route R1: the pseudo-transient iteration in C, ``apt``; route R2: the
same discrete problem assembled and solved directly, ``operator``) and the
closed forms that pin it (``analytic``).  Only the tests, the smoke check and
the benchmark's CPU-baseline leg may import this package; the CUDA library and
its Python binding never do.
"""
