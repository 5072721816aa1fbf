"""B300-native lattice Dirac-operator solver (Wilson twisted-mass/clover and HISQ).

The compute path is the CUDA library built from ``csrc/`` and reached through
the C ABI declared in ``include/lq.h``; ``lib`` is the thin ctypes binding.
"""
