"""Hop-size continuous wavelet transform (CWTH) on GB300.

The transform itself runs in ``libcwth.so`` (hand-written sm_103a CUDA behind
a C ABI declared in ``include/cwth.h``); ``paper_2408_14302_gb300.cwth`` is
the thin ctypes binding and ``paper_2408_14302_gb300.signals`` draws the
seeded synthetic workloads.  Importing this package loads nothing native.
"""

__all__ = ["cwth", "signals"]
