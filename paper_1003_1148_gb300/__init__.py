"""GB300-native (sm_103a) SOP-model overdamped Langevin dynamics.

The simulation runs in the CUDA library ``_lib/libsop.so`` behind the C ABI of
``include/sop.h``; ``sop`` is its ctypes binding and ``synth`` makes seeded
synthetic workloads. Importing this package loads nothing; ``sop.load()``
loads the library and raises if it is missing.
"""
__all__ = ["sop", "synth", "build"]
