"""GB300-native SPH substep with two-way solid coupling (SPHaptics, arXiv 2511.15908).

The compute path is the sm_103a shared library built from ``csrc/`` (C ABI in
``include/sph.h``); :mod:`.sph` is its ctypes binding and :mod:`.scenes` the seeded
synthetic scene generator.
"""
__all__ = ["scenes", "sph"]
