"""GF(2) PLS decomposition, rank, RREF and product on GB300 (sm_103a).

The compute path is the C-ABI library ``libgf2.so`` built from ``csrc/``;
``paper_1006_1744_gb300.gf2`` is its thin ctypes binding. The library is
loaded lazily on first use and a missing build raises immediately: there is no
CPU fallback.
"""
