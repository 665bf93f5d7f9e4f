"""GB300-native loopy belief propagation engine (PGMax's method, arXiv 2202.04110).

* ``workloads``: seeded synthetic factor graphs and inputs (no BP arithmetic).
* ``build``: compiles ``libpgm.so`` (CUDA, sm_103a) in-tree.
* ``binding``: thin ctypes binding of the C ABI in ``include/pgm.h``.
"""
