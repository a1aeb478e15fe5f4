"""GB300-native lattice-Boltzmann phase-field solver (arXiv 1602.07483).

The compute path is the CUDA shared library ``_lib/liblbpf.so`` built from
``csrc/`` for sm_103a; :mod:`.lbpf` is its thin ctypes binding and
:mod:`.workloads` the seeded input recipes.  Importing this package does not load
the library; :func:`lbpf.load` does, and raises when it is missing.
"""
__all__ = ["lbpf", "workloads"]
