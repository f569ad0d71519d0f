"""GB300-native space-time DG-SEM (arXiv:2201.05800): residual, Jv and JFNK slab solves.

The compute path is the CUDA library ``libstdg.so`` (C-ABI declared in
``include/stdg.h``); ``paper_2201_05800_gb300.stdg`` is its thin ctypes
binding.  Importing this package does not load the library; the first call
into ``stdg`` does, and raises if it has not been built.
"""
