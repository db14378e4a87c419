"""GB300-native Newton-step solver for dual-porosity oil-water reservoir
simulation (CPR-FPF preconditioned FGMRES), behind the C ABI of
``include/dpsim.h``.

``paper_1808_04338_gb300.build.build()`` compiles ``libdpsim.so`` for sm_103a;
``paper_1808_04338_gb300.dpsim`` is the ctypes binding.  Nothing is loaded
at import time.
"""
__all__ = ["build", "dpsim"]
