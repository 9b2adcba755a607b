"""Exhaustive finite Kripke evaluation on GB300 (sm_103a).

The compute path is ``libmk`` (C ABI, ``include/mk.h``): a host compiler and
certificate checker in C++ and the census / separation / learned-proposal
kernels in CUDA.  ``paper_2606_15437_gb300.mk`` is the thin ctypes binding
with the same names; ``workloads`` makes the seeded synthetic inputs.
Importing this package loads nothing: the library is loaded on first use.
"""
