"""GB300-native MFV/MFM hydro step (arXiv:2211.12243, §2.3) behind a C ABI.

The CUDA library ``libhydro.so`` (sources in ``csrc/``, declarations in
``include/hydro.h``) holds every kernel of the step; ``hydro`` is its thin
ctypes binding.  ``workloads`` holds the seeded initial-condition generators.
"""
