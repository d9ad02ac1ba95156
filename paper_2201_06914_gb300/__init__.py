"""GB300-native probed (randomized-trace) adjoint-state gradient.

The CUDA path lives in csrc/ and is loaded through `paper_2201_06914_gb300.wp` (a thin
ctypes binding of the C-ABI declared in include/wp.h).  `inputs` builds seeded synthetic
workloads.  Importing the package loads nothing compiled; `wp` raises if the library is
missing.
"""
