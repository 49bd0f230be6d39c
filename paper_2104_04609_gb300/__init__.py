"""GB300-native OSRC-preconditioned PMCHWT solver for acoustic transmission.

Hot path in hand-written CUDA for sm_103a behind the C ABI of
include/osrc_pmchwt.h; ``binding`` is the thin Python marshalling layer,
``inputs`` the seeded synthetic workload generators, ``build`` the in-tree
nvcc build.  Submodules are imported on demand so that ``inputs`` can be used
without loading the CUDA library.
"""
__all__ = ["binding", "inputs", "build"]
