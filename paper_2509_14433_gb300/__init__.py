"""GB300-native sketch-based dynamic connectivity (arXiv 2509.14433).

The compute path is the CUDA library ``libcupc.so`` (C-ABI declared in
``include/cupc.h``); ``paper_2509_14433_gb300.cupc`` is its thin ctypes
binding. Importing this package does not load the library; importing
``paper_2509_14433_gb300.cupc`` does, and fails loudly if it is not built.
"""

__all__ = ["cupc", "workloads"]
