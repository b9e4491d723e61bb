"""GB300-native flux-limited-diffusion (FLD) radiation-energy update.

The compute path is a C-ABI CUDA library (``csrc/``, declared in ``include/fld.h``)
for sm_103a; ``paper_2104_03968_gb300.fld`` is a thin ctypes binding over it.
Importing this package does not load the library; the binding loads it on first use
and raises if it is missing.
"""
__all__ = ["fld", "inputs"]
