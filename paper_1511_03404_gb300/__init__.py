"""rs: LSD radix sort for NVIDIA GB300 (sm_103a).

A from-scratch implementation of the parallel LSD radix sort of Bozidar &
Dobravec, "Comparison of parallel sorting algorithms" (arXiv 1511.03404),
Sec. 2.6: digit histograms, exclusive scans and stable scatters, one pass
per r-bit digit from least to most significant, over 32-bit keys, 32-bit
key-value pairs, 64-bit keys and 64-bit key-value pairs.

The compute path is the CUDA library under ``csrc/`` (C ABI in
``include/rs.h``); ``rs`` is its ctypes binding.
"""
from . import rs  # noqa: F401
from .rs import (RsError, check, load, segmented_sort, sort, status_string,  # noqa: F401
                 workspace)

__all__ = ["rs", "RsError", "check", "load", "segmented_sort", "sort", "status_string",
           "workspace"]
