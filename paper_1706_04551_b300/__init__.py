"""B300-native non-hydrostatic shallow-water step (arXiv:1706.04551).

The compute path is the CUDA library ``libnh.so`` (sources in ``csrc/``, C-ABI declared in
``include/nh.h``); ``nh`` is its thin ctypes binding and ``inputs`` draws the seeded
synthetic workloads.  Importing the package does not load the library; ``nh.load()`` does,
and fails loudly when it is missing.
"""
__all__ = ["inputs", "nh"]
